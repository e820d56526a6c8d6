"""The C ABI from C: include/prtgs.h compiles as C11 and a program linked against libprtgs.so
gets the host-side answers (no GPU needed)."""
import os
import shutil
import subprocess

import pytest

from paper_2408_03538_gb300 import _lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_header_compiles_as_c_and_links(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    so = L.load()._name
    libdir = os.path.dirname(so)
    cuda_lib = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64")
    exe = str(tmp_path / "abi_check")
    cmd = [cc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c", "abi_check.c"), "-o", exe, so,
           f"-Wl,-rpath,{libdir}", f"-Wl,-rpath,{cuda_lib}"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    lines = out.stdout.strip().splitlines()
    assert lines[-1] == "ok"
    import ctypes

    sizes = [int(x) for x in lines[0].split()[1:]]
    assert sizes == [ctypes.sizeof(t) for t in (L.Gaussians, L.BVH, L.TransferParams, L.Camera, L.RenderState,
                                                L.TuneTransfer, L.TuneRelight)]
