"""The library's host-table self-test catches plausible mistakes.

Each case plants one mistake in a temporary copy of the host runtime
(``pma_host.cu``: the neighbour table of the transmission gathers, the
transmission flags of staged bands), links it with the built kernels and
runs ``pma_selftest_tables`` in a child process: a mutant that passes means
the self-test leaves that part of the tables unchecked.  CPU only (no device
is touched).
"""
import os
import subprocess
import sys

import pytest

from paper_2006_14602_gb300 import build as B

SRC = os.path.join(B.CSRC, "pma_host.cu")

MUTANTS = {
    # 2D subdomains: the z offset of the 9 neighbour entries must be 0
    "nb_2d_z_offset": ("per == 27 ? q / 9 - 1 : 0}", "q / 9 - 1}"),
    # the plane stride of a neighbour is pitch x n1, not the pitch
    "nb_plane_stride": ("e.plane = (int)plane;", "e.plane = (int)pitch;"),
    # the shift from this subdomain's local index to the owner's
    "nb_offset_sign": ("const long long c0 = (me.g0[0] - o.g0[0])",
                       "const long long c0 = (o.g0[0] - me.g0[0])"),
    # candidate staged rows of a band's transmission flags
    "band_flag_rows": ("const int cand[4] = {0, 1, sh - 2, sh - 1};\n  int fl = 0;",
                       "const int cand[4] = {0, 2, sh - 2, sh - 1};\n  int fl = 0;"),
}

_RUN = r"""
import ctypes, sys
lib = ctypes.CDLL(sys.argv[1])
lib.pma_selftest_tables.restype = ctypes.c_int32
print(lib.pma_selftest_tables())
"""


@pytest.fixture(scope="module")
def kernels_obj():
    B.build()
    return os.path.join(B.OUT, "pma_kernels.o")


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_selftest_catches_planted_mistake(name, kernels_obj, tmp_path):
    a, b = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(a) == 1, name
    mut = tmp_path / "pma_host.cu"
    mut.write_text(src.replace(a, b))
    obj = tmp_path / "pma_host.o"
    lib = tmp_path / "libpma_mut.so"
    nvcc = B._nvcc()
    flags = B.ARCH + ["-O1", "-std=c++17", "-Xcompiler", "-fPIC", "-I", B.INCLUDE, "-I", B.CSRC]
    r = subprocess.run([nvcc] + flags + ["-c", str(mut), "-o", str(obj)], capture_output=True,
                       text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([nvcc] + B.ARCH + ["-shared", "-o", str(lib), str(obj), kernels_obj],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([sys.executable, "-c", _RUN, str(lib)], capture_output=True, text=True)
    assert out.returncode == 0, out.stderr
    assert int(out.stdout.strip()) > 0, "mutant %s passed the self-test" % name
