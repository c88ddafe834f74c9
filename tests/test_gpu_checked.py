"""The checked build (libn2f_checked.so, the sources compiled with N2F_CHECKED): its kernels test
every global-memory index they compute against the extent of the tensor it addresses and count
the ones out of range instead of accessing them. Every kernel family runs on ragged and odd
shapes in a fresh process that loads the checked library, and no index may fall outside."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_checked_build_finds_no_index_out_of_range():
    import __graft_entry__  # noqa: F401  (repository root on sys.path)
    from paper_2108_10209_gb300 import build
    build.build(checked=True)
    env = dict(os.environ, N2F_LIBRARY="checked")
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_workload.py")], env=env,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stderr[-4000:]
    line = [l for l in r.stdout.splitlines() if l.startswith("{")][-1]
    res = json.loads(line)
    print(res)
    assert res["failures"] == 0, res
    assert len(res["ran"]) == 5
