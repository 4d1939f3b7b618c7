"""The boundary from plain C: tests/c/abi_smoke.c includes only radtex.h and
the CUDA runtime, is compiled with gcc as C99 and linked against
libradtex.so.  On the CPU it calls the host-only entry points; on a GPU it
creates a context and a constant texture through the C ABI and checks that
shading returns the constant exactly."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2301_01719_gb300")


@pytest.fixture(scope="module")
def c_program(tmp_path_factory):
    from paper_2301_01719_gb300 import build

    try:
        nvcc = build.nvcc()
    except RuntimeError:
        pytest.skip("no CUDA toolkit")
    build.build()
    cuda = os.path.dirname(os.path.dirname(nvcc))
    libdir = next((os.path.join(cuda, d) for d in ("lib64", "lib", "targets/sbsa-linux/lib",
                                                    "targets/x86_64-linux/lib")
                   if os.path.exists(os.path.join(cuda, d, "libcudart.so"))), None)
    if libdir is None:
        pytest.skip("no libcudart.so next to nvcc")
    exe = str(tmp_path_factory.mktemp("cabi") / "abi_smoke")
    cmd = ["gcc", "-std=c99", "-Wall", "-Werror", "-O1", os.path.join(ROOT, "tests", "c", "abi_smoke.c"),
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include"), "-L", PKG, "-lradtex",
           "-L", libdir, "-lcudart", f"-Wl,-rpath,{PKG}", f"-Wl,-rpath,{libdir}", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    return exe


def test_c_program_links_and_calls_host_entry_points(c_program):
    r = subprocess.run([c_program], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    lines = r.stdout.splitlines()
    assert lines[0].startswith("status 1 ") and "argument" in lines[0].lower()
    assert int(lines[1].split()[-1]) > 0


@pytest.mark.gpu
def test_c_program_shades_a_constant_texture(c_program):
    r = subprocess.run([c_program, "gpu"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "gpu ok" in r.stdout, r.stdout + r.stderr
