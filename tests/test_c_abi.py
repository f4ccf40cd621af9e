"""The C-ABI from plain C: tests/c/abi_check.c is compiled with gcc as C99
against include/xf.h, linked to the library and run (no device needed)."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_header_and_library_work_from_c99():
    from paper_2403_05910_b300 import build
    lib = build.build()
    exe = os.path.join(ROOT, "tests", "c", "abi_check")   # git-ignored build product
    src = os.path.join(ROOT, "tests", "c", "abi_check.c")
    cmd = ["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), src,
           "-o", exe, "-L", os.path.dirname(lib), "-lxf",
           "-Wl,-rpath," + os.path.dirname(lib)]
    subprocess.check_call(cmd)
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0, (out.returncode, out.stdout, out.stderr)
    assert out.stdout.startswith("ok")
