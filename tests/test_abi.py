"""CPU-only checks of the C ABI boundary: the library builds for sm_103a,
loads, and exports every function include/*.h declares; the Python binding
covers the same names; host-side argument checks work without a GPU."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names += re.findall(r"^RS_API\s+[\w\s\*]+?\b(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1206_3511_gb300 import _build, _lib

    _build.build()
    return ctypes.CDLL(_lib.LIB_PATH)


def test_header_declares_entry_points():
    names = _declared()
    assert "rs_sort_u32" in names and "rs_sort_u64" in names and "rs_get_status" in names
    assert len(names) >= 15


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_python_binding_names_match_header():
    from paper_1206_3511_gb300 import _lib

    assert set(_declared()) == set(_lib.SIGNATURES), set(_declared()) ^ set(_lib.SIGNATURES)
    for n in _declared():
        assert callable(getattr(_lib, n)), n


def test_host_side_queries_need_no_gpu(lib):
    from paper_1206_3511_gb300 import _lib

    _lib.load()
    assert _lib.rs_version() >= 100
    assert "RS_ERR_WORKSPACE" in _lib.rs_status_string(2)
    ws = _lib.rs_workspace_bytes(0, 4, 0, 10**8, 32, 0, 0)
    # header + counts + two status arrays + one 400 MB ping-pong buffer
    assert 400_000_000 < ws < 500_000_000
    assert _lib.rs_workspace_bytes(0, 4, 0, 10**8, 33, 0, 0) == 0   # key_bits above the key width
    assert _lib.rs_workspace_bytes(0, 3, 0, 10, 0, 0, 0) == 0
    cfg = _lib.rs_default_config(4, 0, 10**8)
    assert cfg.digit_bits == 8 and cfg.as_tuple() == (8, 256, 36)
    # small u32 keys-only sorts take the larger-tile shape; other key types do not
    assert _lib.rs_default_config(4, 0, 10**6).as_tuple() == (8, 512, 15)
    assert _lib.rs_default_config(4, 0, (1 << 22) + 1).as_tuple() == (8, 256, 36)
    assert _lib.rs_default_config(4, 1, 10**6).as_tuple() == (8, 256, 20)
    assert _lib.rs_config_count(4, 0) >= 8
    seen = {_lib.rs_config_get(4, 0, i).as_tuple() for i in range(_lib.rs_config_count(4, 0))}
    assert len(seen) == _lib.rs_config_count(4, 0)


def test_argument_errors_are_returned_before_any_launch(lib):
    from paper_1206_3511_gb300 import _lib

    _lib.load()
    fake = 1 << 40  # never dereferenced: every call below fails validation first
    # vals_in without vals_out
    assert _lib.rs_sort_u32(fake, fake + 4096, fake, None, 16, 32, fake, 1 << 20, 0) == 1
    # key_bits out of range
    assert _lib.rs_sort_u32(fake, fake + 4096, None, None, 16, 33, fake, 1 << 20, 0) == 1
    # misaligned / missing workspace
    assert _lib.rs_sort_u32(fake, fake + 4096, None, None, 16, 32, fake + 8, 1 << 20, 0) == 2
    assert _lib.rs_sort_u32(fake, fake + 4096, None, None, 16, 32, None, 1 << 20, 0) == 2
    # workspace too small
    assert _lib.rs_sort_u32(fake, fake + 4096, None, None, 1000, 32, fake + (1 << 30), 64, 0) == 2
    # partial overlap of input and output
    assert _lib.rs_sort_u32(fake, fake + 8, None, None, 16, 32, fake + (1 << 30), 1 << 20, 0) == 1
    # n above the single-sort limit
    assert _lib.rs_sort_u32(fake, fake + 4096, None, None, (1 << 30) + 1, 32, fake, 1 << 20, 0) == 1
    # n == 0 is a no-op
    assert _lib.rs_sort_u32(None, None, None, None, 0, 32, fake, 1 << 20, 0) == 0
    # a configuration that is not compiled
    assert _lib.rs_sort_u32_ex(fake, fake + 4096, None, None, 16, 32, fake, 1 << 20, 0, (8, 256, 3)) == 9


def test_argument_errors_of_the_other_entry_points(lib):
    """Bucket, segmented, typed, bucket-count and server entry points reject
    bad arguments on the host, before any CUDA call (so this runs without a
    GPU)."""
    from paper_1206_3511_gb300 import _lib

    _lib.load()
    fake = 1 << 40
    big_ws = fake + (1 << 30)
    # bucket sort: values without outputs, overlap, misaligned keys, workspace
    assert _lib.bs_sort_u32(fake, fake + 4096, fake, None, 16, 0, 99, 0, big_ws, 1 << 30, 0) == 1
    assert _lib.bs_sort_u32(fake, fake + 8, None, None, 16, 0, 99, 0, big_ws, 1 << 30, 0) == 1
    assert _lib.bs_sort_u64(fake + 4, fake + 4096, None, None, 16, 0, 99, 0, big_ws, 1 << 30, 0) == 1
    assert _lib.bs_sort_u32(fake, fake + 4096, None, None, 16, 0, 99, 0, None, 1 << 30, 0) == 2
    assert _lib.bs_sort_u32(fake, fake + 4096, None, None, 1000, 0, 99, 0, big_ws, 64, 0) == 2
    assert _lib.bs_sort_u32(fake, fake + 4096, None, None, 16, 0, 99, (1 << 32) + 1, big_ws, 1 << 30, 0) == 1
    assert _lib.bs_sort_u32(None, None, None, None, 0, 0, 99, 0, big_ws, 1 << 30, 0) == 0  # n == 0
    # segmented: key_bits, workspace, a shape that is not compiled
    assert _lib.rs_sort_segmented_u32(fake, fake + 4096, None, None, fake, 3, 16, 33, big_ws, 1 << 30, 0) == 1
    assert _lib.rs_sort_segmented_u32(fake, fake + 4096, None, None, fake, 3, 16, 32, None, 1 << 30, 0) == 2
    assert _lib.rs_sort_segmented_u32(fake, fake + 4096, None, None, fake, 3, 1000, 32, big_ws, 64, 0) == 2
    assert _lib.rs_sort_segmented_u32_ex(fake, fake + 4096, None, None, fake, 3, 16, 32, big_ws, 1 << 30, 0,
                                         (7, 256, 18)) == 9
    assert _lib.rs_sort_segmented_u32(fake, fake + 4096, None, None, fake, 0, 0, 32, big_ws, 1 << 30, 0) == 0
    # typed keys: kind, width
    assert _lib.rs_sort_typed(3, 4, 0, fake, fake + 4096, None, None, 16, big_ws, 1 << 30, 0) == 1
    assert _lib.rs_sort_typed(1, 2, 0, fake, fake + 4096, None, None, 16, big_ws, 1 << 30, 0) == 1
    assert _lib.rs_sort_typed(2, 8, 1, fake, fake + 8, None, None, 16, big_ws, 1 << 30, 0) == 1  # overlap
    # bucket counts: bounds, bucket count, output pointer, workspace
    assert _lib.bs_bucket_counts_u32(fake, 16, 9, 5, 4, fake + 4096, big_ws, 4096, 0) == 1
    assert _lib.bs_bucket_counts_u32(fake, 16, 0, 99, 0, fake + 4096, big_ws, 4096, 0) == 1
    assert _lib.bs_bucket_counts_u32(fake, 16, 0, 99, 4, None, big_ws, 4096, 0) == 1
    assert _lib.bs_bucket_counts_u64(fake, 16, 0, 99, 4, fake + 4096, big_ws, 64, 0) == 2
    # server: configuration
    bad = _lib.RsServerConfig(None, 1 << 20, 0, 4, 8, 0)
    assert _lib.rs_server_create(bad)[0] == 1
    bad = _lib.RsServerConfig(fake, 1 << 20, 0, 0, 8, 0)  # no streams
    assert _lib.rs_server_create(bad)[0] == 1
    bad = _lib.RsServerConfig(fake + 8, 1 << 20, 0, 4, 8, 0)  # misaligned pool
    assert _lib.rs_server_create(bad)[0] == 1


def test_host_buffer_sorts_size_and_reject_bad_arguments(lib):
    """The host-buffer sorts: dev_buf holds the workspace, the keys and the
    values; arguments that need no CUDA call are checked first."""
    from paper_1206_3511_gb300 import _lib

    _lib.load()
    n = 10**6
    ws = _lib.rs_workspace_bytes(0, 4, 0, n, 32, 0, 1)
    assert _lib.rs_host_sort_bytes(0, 4, 0, n, 32, 0) >= ws + 4 * n
    assert _lib.rs_host_sort_bytes(0, 8, 1, n, 0, 0) >= _lib.rs_workspace_bytes(0, 8, 1, n, 0, 0, 1) + 12 * n
    assert _lib.rs_host_sort_bytes(1, 4, 0, n, 0, 0) >= _lib.rs_workspace_bytes(1, 4, 0, n, 0, 0, 1) + 4 * n
    assert _lib.rs_host_sort_bytes(0, 4, 0, n, 33, 0) == 0
    assert _lib.rs_host_sort_bytes(2, 4, 0, n, 0, 0) == 0
    assert _lib.rs_host_sort_bytes(1, 4, 0, n, 0, (1 << 32) + 1) == 0
    h = ctypes.create_string_buffer(1 << 16)
    a = ctypes.addressof(h)
    a += (-a) % 16
    fake_dev = 1 << 40
    # values without outputs, key_bits, n above the limit, null keys
    assert _lib.rs_sort_host_u32(a, a + 4096, a, None, 16, 32, fake_dev, 1 << 30, 0) == 1
    assert _lib.rs_sort_host_u32(a, a + 4096, None, None, 16, 33, fake_dev, 1 << 30, 0) == 1
    assert _lib.rs_sort_host_u32(a, a + 4096, None, None, (1 << 30) + 1, 32, fake_dev, 1 << 30, 0) == 1
    assert _lib.rs_sort_host_u64(None, a, None, None, 16, 0, fake_dev, 1 << 30, 0) == 1
    # misaligned keys, partial overlap of keys in and out, keys over values
    assert _lib.rs_sort_host_u64(a + 4, a + 4096, None, None, 16, 0, fake_dev, 1 << 30, 0) == 1
    assert _lib.rs_sort_host_u32(a, a + 8, None, None, 16, 32, fake_dev, 1 << 30, 0) == 1
    assert _lib.rs_sort_host_u32(a, a + 4096, a + 2048, a + 32, 16, 32, fake_dev, 1 << 30, 0) == 1
    # n == 0 is a no-op
    assert _lib.rs_sort_host_u32(None, None, None, None, 0, 32, None, 0, 0) == 0
    # bucket: bucket count above 2^32, values without outputs, overlap
    assert _lib.bs_sort_host_u32(a, a + 4096, None, None, 16, 0, 99, (1 << 32) + 1, fake_dev, 1 << 30, 0) == 1
    assert _lib.bs_sort_host_u32(a, a + 4096, a, None, 16, 0, 99, 0, fake_dev, 1 << 30, 0) == 1
    assert _lib.bs_sort_host_u64(a, a + 8, None, None, 16, 0, 99, 0, fake_dev, 1 << 30, 0) == 1
    assert _lib.bs_sort_host_u64(None, None, None, None, 0, 0, 99, 0, None, 0, 0) == 0


def test_segmented_host_sort_rejects_bad_arguments(lib):
    from paper_1206_3511_gb300 import _lib

    _lib.load()
    n, nseg = 10**6, 1000
    assert _lib.rs_segmented_host_bytes(4, 0, n, nseg, 32) >= (
        _lib.rs_segmented_workspace_bytes(4, 0, n, nseg, 32) + 4 * n + 8 * (nseg + 1))
    assert _lib.rs_segmented_host_bytes(4, 0, n, nseg, 33) == 0
    h = ctypes.create_string_buffer(1 << 16)
    a = ctypes.addressof(h)
    a += (-a) % 16
    offs = a + 8192
    fake_dev = 1 << 40
    f = _lib.rs_sort_segmented_host_u32
    assert f(a, a + 4096, None, None, offs, 3, 16, 33, fake_dev, 1 << 30, 0, None) == 1      # key_bits
    assert f(a, a + 4096, a + 6000, None, offs, 3, 16, 32, fake_dev, 1 << 30, 0, None) == 1  # values
    assert f(a, a + 4096, None, None, None, 3, 16, 32, fake_dev, 1 << 30, 0, None) == 1      # no offsets
    assert f(a, a + 4096, None, None, offs + 4, 3, 16, 32, fake_dev, 1 << 30, 0, None) == 1  # misaligned
    assert f(a, a + 4096, None, None, a + 4104, 3, 16, 32, fake_dev, 1 << 30, 0, None) == 1  # offsets in output
    assert f(a, a + 8, None, None, offs, 3, 16, 32, fake_dev, 1 << 30, 0, None) == 1         # keys overlap
    assert f(None, None, None, None, None, 0, 0, 32, None, 0, 0, None) == 0                  # nothing to sort
