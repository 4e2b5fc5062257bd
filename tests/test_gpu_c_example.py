"""The C example (examples/slab_dose.c) runs a dose calculation through the
C ABI alone and reports a balanced energy ledger."""
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
