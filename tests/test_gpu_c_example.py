"""The C examples run through the C ABI alone: examples/slab_dose.c a dose
calculation with a balanced energy ledger, examples/serve_requests.c
several requests served side by side, each finishing with its own balanced
ledger."""
import re
import subprocess

import pytest

from tests.test_abi import build_c_example

pytestmark = pytest.mark.gpu


def test_c_example_runs(tmp_path):
    exe = build_c_example(tmp_path)
    r = subprocess.run([exe, "1000000"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    print(r.stdout)
    assert "histories 1000000" in r.stdout
    bal = float(re.search(r"energy balance \(relative\) (\S+)", r.stdout).group(1))
    assert abs(bal) < 1e-5
    sig = float(re.search(r"sigma/Dmax (\S+) %", r.stdout).group(1))
    assert 0 < sig < 20


def test_c_serving_example_runs(tmp_path):
    exe = build_c_example(tmp_path, "serve_requests")
    r = subprocess.run([exe, "8"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    print(r.stdout)
    rows = [ln.split() for ln in r.stdout.splitlines()[1:] if ln.strip()]
    assert sorted(int(x[0]) for x in rows) == list(range(8))
    for x in rows:
        assert int(x[2]) == (200000 if int(x[0]) % 2 == 0 else 2000000)
        assert abs(float(x[5])) < 1e-5
