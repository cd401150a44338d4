"""The environment switches, each read once per process, so every case runs
in a child process: RS_DIGIT_BITS changes the default digit width (and the
sort stays exact), RS_CHECKED=1 adds the device order check to every plain
sort (one more launch, status still RS_OK on correct output), and
RS_SPIN_LIMIT is accepted.  Results are compared with numpy's stable sort of
the same keys (the oracle's radix sort is pinned equal to it)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys, numpy as np, torch
sys.path.insert(0, ROOT)
import paper_1206_3511_gb300 as rs, synth
from tests._util import to_dev, from_dev
rs.load()
cfg = rs.rs_default_config(4, 0, 10**8).as_tuple()
print("default", cfg[0], cfg[1], cfg[2])
for n in (3000, 2_000_003):
    keys = synth.u32(n, 77, 0)
    kd = to_dev(keys)
    ws = rs.workspace(rs.rs_workspace_bytes(0, 4, 0, n, 32, 0, 0))
    out = torch.empty_like(kd)
    l0 = rs.rs_launch_count()
    assert rs.rs_sort_u32(kd, out, None, None, n, 32, ws, ws.numel()) == 0
    torch.cuda.synchronize()
    print("launches", n, rs.rs_launch_count() - l0)
    assert rs.get_status(ws) == 0
    assert np.array_equal(from_dev(out, np.uint32), np.sort(keys, kind="stable"))
    bkeys = synth.keys_u32(n, 6, seed=3)
    ok, _ = rs.bucket_sort(to_dev(bkeys))
    torch.cuda.synchronize()
    assert np.array_equal(from_dev(ok, np.uint32), np.sort(bkeys, kind="stable"))
print("ok")
'''.replace("ROOT", repr(ROOT))


def _child(env_extra):
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    lines = dict((ln.split()[0], ln.split()[1:]) for ln in r.stdout.splitlines() if ln and ln.split()[0] != "launches")
    launches = {int(ln.split()[1]): int(ln.split()[2]) for ln in r.stdout.splitlines() if ln.startswith("launches")}
    assert "ok" in lines
    return lines, launches


def test_defaults_then_switches():
    base, base_launches = _child({"RS_DIGIT_BITS": "", "RS_CHECKED": "", "RS_SPIN_LIMIT": ""})
    assert base["default"][0] == "8"
    wide, _ = _child({"RS_DIGIT_BITS": "9"})
    assert wide["default"][0] == "9"
    _, checked_launches = _child({"RS_CHECKED": "1", "RS_SPIN_LIMIT": "100000"})
    for n, k in base_launches.items():
        assert checked_launches[n] == k + 1, (n, k, checked_launches[n])
