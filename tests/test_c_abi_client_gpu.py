"""The C ABI from a plain C program (tests/c_abi_client.c): compiled with gcc
against include/latch.h, liblatch.so and the CUDA runtime only, then run on the
GPU.  It extracts a small image's descriptors, matches the set against itself on
both paths and checks an argument error."""
import os
import subprocess

import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_c_client(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1609_03986_gb300 import build
    lib = build.build()
    cuda = build._cuda_home()
    libdir = os.path.dirname(lib)
    exe = str(tmp_path / "c_abi_client")
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I" + os.path.join(ROOT, "include"),
                           "-I" + os.path.join(cuda, "include"), os.path.join(HERE, "c_abi_client.c"), "-o", exe,
                           "-L" + libdir, "-llatch", "-L" + os.path.join(cuda, "lib64"), "-lcudart",
                           "-Wl,-rpath," + libdir + ":" + os.path.join(cuda, "lib64")])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == "ok"
