"""The C ABI from plain C: tests/c_abi_check.c includes include/hp.h as C99
(no C++ in the header), links against libhp.so and drives the host-side calls
(create, add_stage, set_output, schedule_set, group info, bounds inference,
errors, destroy) with no Python or torch in the process."""

import os
import shutil
import subprocess

import pytest

import __graft_entry__
from paper_2012_07145_gb300 import hp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_plain_c_program_drives_the_library(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    __graft_entry__.build()
    libdir = os.path.dirname(hp.LIB_PATH)
    exe = str(tmp_path / "c_abi_check")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        os.path.join(ROOT, "tests", "c_abi_check.c"), "-o", exe, "-L", libdir, "-lhp",
                        "-Wl,-rpath," + libdir], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
