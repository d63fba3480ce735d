"""C-ABI checks that need no GPU: the library builds, loads and exports every
entry point of include/pma.h; the ctypes structs match the C layout; the
library refuses to run without a device (no CPU fallback)."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

from paper_2006_14602_gb300 import build as B
from paper_2006_14602_gb300 import pma

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pma.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return pma.load()


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pma_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_entry_point_is_exported(lib):
    names = _declared()
    assert len(names) >= 19
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(pma.exported_symbols()) == names
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True)
    exported = set(re.findall(r" T (pma_\w+)", out.stdout))
    assert set(names) <= exported


_LAYOUT_PROBE = r"""
#include <stdio.h>
#include <stddef.h>
#include "pma.h"
#define F(T, f) printf(#T "." #f " %zu\n", offsetof(T, f));
int main(void) {
  printf("pma_grid %zu\npma_term %zu\npma_monitor %zu\npma_decomp %zu\n"
         "pma_params %zu\npma_info %zu\npma_stats %zu\n", sizeof(pma_grid), sizeof(pma_term),
         sizeof(pma_monitor), sizeof(pma_decomp), sizeof(pma_params), sizeof(pma_info),
         sizeof(pma_stats));
  F(pma_grid, lo) F(pma_grid, hi) F(pma_term, amp) F(pma_term, c)
  F(pma_monitor, base) F(pma_monitor, term) F(pma_decomp, overlap)
  F(pma_decomp, exchange_every)
  F(pma_params, max_steps) F(pma_params, precision) F(pma_info, status)
  F(pma_info, latency_us) F(pma_stats, sweep_kernel_launches) F(pma_stats, combine_ms)
  return 0;
}
"""


def test_struct_layout_matches_header():
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "probe.c")
        open(c, "w").write(_LAYOUT_PROBE)
        exe = os.path.join(d, "probe")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        lines = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    got = dict(l.split() for l in lines.strip().splitlines())
    S = {"pma_grid": pma.pma_grid, "pma_term": pma.pma_term, "pma_monitor": pma.pma_monitor,
         "pma_decomp": pma.pma_decomp, "pma_params": pma.pma_params, "pma_info": pma.pma_info,
         "pma_stats": pma.pma_stats}
    for k, v in got.items():
        if "." in k:
            s, f = k.split(".")
            assert getattr(S[s], f).offset == int(v), k
        else:
            assert C.sizeof(S[k]) == int(v), k


def test_status_strings_and_version(lib):
    assert pma.pma_abi_version() == 2
    assert pma.pma_status_str(pma.PMA_ERR_TANGLED) == "mesh tangled"
    assert pma.pma_status_str(12345) == "unknown status"
    assert isinstance(pma.pma_last_error(), str)


def test_no_device_means_loud_failure(lib):
    """Without a GPU the library reports a CUDA error; nothing runs on the CPU."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    st, h = pma.pma_create(0, 0, 0)
    assert st == pma.PMA_ERR_CUDA and not h.value
    assert pma.pma_last_error()


def test_missing_library_raises(tmp_path, monkeypatch):
    monkeypatch.setattr(pma, "_lib", None)
    with pytest.raises(RuntimeError):
        pma.load(str(tmp_path / "nope.so"))
    monkeypatch.setattr(pma, "_lib", None)


def test_problem_marshalling():
    from paper_2006_14602_gb300 import workloads as W
    g, m, d, p = pma.to_structs(W.config2("sine", "fp32"))
    assert (g.dim, list(g.n)) == (2, [257, 257, 1])
    assert m.kind == 0 and m.nterms == 1 and m.term[0].type == 2
    assert m.term[0].axis == 1 and m.term[0].along == 0 and m.term[0].a == 0.25
    assert list(d.parts) == [4, 4, 1] and d.overlap == 8
    assert p.precision == 0 and p.max_steps == 2000
    with pytest.raises(ValueError):
        pma.to_structs(W.small_case().replace(rhs="root"))


def test_host_tables_selftest(lib):
    """The library's host-only self-test of the tables its kernels index:
    neighbour entries of the transmission gathers against the owners from
    the decomposition's core boundaries, the staged bands' transmission
    flags, and the work items' tiling and shared-memory / TMA limits."""
    n = pma.pma_selftest_tables()
    assert n == 0, pma.pma_last_error()
