"""The library used from C through include/zkntt.h alone (tests/c_abi/ntt_file.c):
the program compiles against the header, links libzkntt.so and the CUDA
runtime, and (on a GPU) runs a transform whose output equals the oracle's."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import cpu
from oracle import field as fld
from workloads import uniform_elements

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


@pytest.fixture(scope="module")
def program(tmp_path_factory):
    from paper_2509_22684_gb300 import build
    lib = build.build()
    libdir = os.path.dirname(lib)
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path_factory.mktemp("c_abi") / "ntt_file")
    cmd = [cc, "-std=c11", "-Wall", "-Werror", os.path.join(ROOT, "tests", "c_abi", "ntt_file.c"),
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(CUDA, "include"),
           "-L", libdir, "-lzkntt", "-L", os.path.join(CUDA, "lib64"), "-lcudart",
           f"-Wl,-rpath,{libdir}", f"-Wl,-rpath,{os.path.join(CUDA, 'lib64')}", "-o", exe]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    return exe


def test_c_program_builds_and_host_checks_pass(program):
    res = subprocess.run([program, "check"], capture_output=True, text=True, timeout=120)
    assert res.returncode == 0, res.stderr
    assert "host checks ok" in res.stdout


@pytest.mark.gpu
@pytest.mark.parametrize("F,L,direction", [(fld.BLS12_381, 12, 0), (fld.BN254, 16, 1),
                                           (fld.BLS12_377, 18, 0)],
                         ids=lambda v: getattr(v, "name", str(v)))
def test_c_program_transform_matches_oracle(program, tmp_path, F, L, direction):
    X = uniform_elements(F.r, 1 << L, 9000 + L)
    src, dst = tmp_path / "in.bin", tmp_path / "out.bin"
    X.astype("<u4").tofile(src)
    fid = fld.FIELD_IDS[F.name]
    res = subprocess.run([program, "run", str(fid), str(L), str(direction), str(src), str(dst)],
                         capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr
    got = np.fromfile(dst, dtype="<u4").reshape(-1, 8)
    want = cpu.ntt(F, X, inverse=bool(direction))
    assert np.array_equal(got, want)
