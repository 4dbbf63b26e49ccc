"""The boundary is a plain C ABI: a C program (tests/c/consumer.c) that
includes only include/spfhe.h and links libspfhe.so plans an Alg. 1 merge,
asks the rotation-base tuner, and gets a malformed CSR refused, with results
equal to the oracle planner's.  Host-side entry points only, so no GPU."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import spmspm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def consumer(tmp_path_factory):
    from paper_2604_11659_gb300 import build
    lib = build.build()
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("no C compiler")
    libdir = os.path.dirname(lib)
    exe = str(tmp_path_factory.mktemp("c") / "consumer")
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", os.path.join(ROOT, "tests", "c", "consumer.c"),
                    "-I", os.path.join(ROOT, "include"), "-L", libdir, "-lspfhe", "-Wl,-rpath," + libdir, "-o", exe],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return out.splitlines()


def test_c_program_plans_like_the_oracle(consumer):
    A = np.zeros((3, 4))
    A[0, 0], A[0, 3], A[2, 1], A[2, 3] = 1, 1, 1, 1
    B = np.zeros((4, 2))
    B[0, 0], B[3, 0], B[1, 1] = 1, 1, 1
    Aip, Aix, _ = spmspm.dense_to_csr(A)
    Bip, Bix, _ = spmspm.dense_to_csc(B)
    want = ["match %d %d %d %d %d" % (m.i, m.j, m.k, m.a_pos, m.b_pos)
            for m in spmspm.alg1_matches(Aip, Aix, Bip, Bix, 3, 2)]
    assert [ln for ln in consumer if ln.startswith("match")] == want


def test_c_program_tuner_and_errors(consumer):
    base = [ln for ln in consumer if ln.startswith("base")]
    assert len(base) == 1
    b = int(base[0].split()[1])
    assert b >= 2 and b & (b - 1) == 0
    bad = [ln for ln in consumer if ln.startswith("bad")][0]
    assert bad.startswith("bad -1 ") and "out of range" in bad
    assert "classes 14 ntt_fwd" in consumer
