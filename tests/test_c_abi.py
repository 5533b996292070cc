"""The boundary as a C client sees it: tests/c/abi_check.c, a C99 program that
includes include/lb.h and links the library, checks the host-side behaviour the
header states (argument validation, NULL handling, status strings). No GPU work."""
import os
import shutil
import subprocess

import pytest

from paper_1008_2865_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c99_client_compiles_links_and_passes(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib = libbuild.build()
    exe = str(tmp_path / "abi_check")
    cmd = [cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
           "-I" + os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c", "abi_check.c"),
           "-L" + os.path.dirname(lib), "-llbsc", "-Wl,-rpath," + os.path.dirname(lib), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "abi_check: ok" in r.stdout


@pytest.mark.gpu
def test_c99_client_runs_a_lattice_on_the_gpu(tmp_path):
    """tests/c/abi_run.c: init from host memory, 200 steps, trace, energy, fields,
    save at t = 100 and resume, all through the C ABI."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lib = libbuild.build()
    exe = str(tmp_path / "abi_run")
    cmd = [cc, "-std=c99", "-O2", "-Wall", "-Wextra", "-Werror", "-I" + os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c", "abi_run.c"), "-L" + os.path.dirname(lib), "-llbsc",
           "-Wl,-rpath," + os.path.dirname(lib), "-lm", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "abi_run: ok" in r.stdout
