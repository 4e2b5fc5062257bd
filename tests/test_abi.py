"""The C ABI library builds for sm_103a, loads, and exports every entry point
declared in include/gdpm.h.  No compute calls: this runs without a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1107_3355_gb300 import build as B
from paper_1107_3355_gb300 import gdpm as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gdpm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gdpm_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["gdpm_phantom_create", "gdpm_tables_build", "gdpm_source_set", "gdpm_simulate",
              "gdpm_request_submit", "gdpm_request_poll", "gdpm_strerror"]:
        assert n in names
    assert sorted(G.EXPORTED) == names


def test_library_builds_and_exports_every_symbol():
    path = B.build()
    lib = ctypes.CDLL(path)
    for n in declared_functions():
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (gdpm_\w+)", out))
    assert set(declared_functions()) <= exported


def test_checked_build_exports_the_same_symbols():
    path = B.build(checked=True)
    assert path.endswith("libgdpm_checked.so")
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    assert set(declared_functions()) <= set(re.findall(r"\bT (gdpm_\w+)", out))


def build_c_example(out_dir, name="slab_dose"):
    """Compile examples/<name>.c with plain gcc against the header and
    libgdpm.so: the C ABI needs neither Python nor PyTorch."""
    lib = B.build()
    exe = os.path.join(str(out_dir), name)
    subprocess.check_call(["gcc", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "examples", name + ".c"), "-L", os.path.dirname(lib),
                           "-lgdpm", "-lm", "-Wl,-rpath," + os.path.dirname(lib), "-o", exe])
    return exe


@pytest.mark.parametrize("name", ["slab_dose", "serve_requests"])
def test_c_example_compiles_and_links(tmp_path, name):
    assert os.access(build_c_example(tmp_path, name), os.X_OK)


def test_strerror_needs_no_device():
    assert G.gdpm_strerror(G.GDPM_E_QUEUE_OVERFLOW) == "secondary particle queue overflow"
    assert G.gdpm_strerror(0) == "ok"
    assert "out of range" in G.gdpm_strerror(G.GDPM_E_BOUNDS)


def test_product_path_refuses_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError):
        G.gdpm_context_create(0)


def test_build_targets_sm103a():
    assert "arch=compute_103a,code=sm_103a" in " ".join(B.ARCH)
