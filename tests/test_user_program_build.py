"""The user-program SDK builds on the CPU (nvcc cross-compiles for
sm_103a): the example programs compile against include/trees_program.cuh
with the public include directory alone on the include path and export
their trees_program_fn launchers; the job record carries one (no kernel runs
here)."""
import ctypes
import os
import subprocess

import paper_1608_00571_b300 as T
from paper_1608_00571_b300 import build as tbuild

EXAMPLES = os.path.join(os.path.dirname(os.path.abspath(T.__file__)), "examples")


def test_example_program_builds_and_exports_its_launcher(tmp_path):
    so = tbuild.build_program(os.path.join(EXAMPLES, "chunk_sum.cu"), str(tmp_path / "libcs.so"))
    out = subprocess.check_output(["nm", "-D", "--defined-only", so], text=True)
    assert any(line.split()[-1] == "trees_chunk_sum" for line in out.splitlines() if line.strip())
    fn = ctypes.CDLL(so).trees_chunk_sum
    job = T.make_job(T.TREES_PROG_USER, user_program=fn, user_type=1, user_a0=3, user_a1=9,
                     user_ptr=(1234,), user_val=(4096, 8))
    assert job.user_program == ctypes.cast(fn, ctypes.c_void_p).value
    assert (job.user_type, job.user_a0, job.user_a1, job.user_ptr[0], job.user_val[1]) == (1, 3, 9, 1234, 8)


def test_sdk_needs_only_the_public_include_directory(tmp_path):
    # a copy of include/ and the example in a scratch tree: nothing of the library's sources is reachable
    import shutil
    root = os.path.dirname(os.path.dirname(os.path.abspath(T.__file__)))
    inc = tmp_path / "include"
    shutil.copytree(os.path.join(root, "include"), inc)
    src = tmp_path / "nqueens.cu"
    shutil.copy(os.path.join(EXAMPLES, "nqueens.cu"), src)
    so = tmp_path / "libnq.so"
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                           "-Xcompiler", "-fPIC", "-shared", "-I", str(inc), str(src), "-o", str(so)],
                          cwd=str(tmp_path))
    out = subprocess.check_output(["nm", "-D", "--defined-only", str(so)], text=True)
    assert any(line.split()[-1] == "trees_nqueens_program" for line in out.splitlines() if line.strip())
