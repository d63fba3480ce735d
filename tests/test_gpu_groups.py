"""Request groups (PMA_OPT_GROUPS, off by default): the requests of a kernel
class split into two groups whose sweep and finish chains run on two
streams.  Requests are
independent, so every mesh must be bitwise the same with one group or two,
with and without CUDA graphs, and the sweep timing must cover the groups'
overlapping launches."""
import numpy as np
import pytest

from paper_2006_14602_gb300 import pma
from paper_2006_14602_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    from paper_2006_14602_gb300 import build
    build.build()
    pma.load()


def _batch():
    probs = W.config4(seed=21, count=14, max_steps=90, size_range=(17, 160))
    probs += [p.replace(precision="fp64") for p in W.config4(seed=22, count=5, max_steps=70,
                                                             size_range=(17, 90))]
    probs += [W.small_case(3, 19, parts=(2, 2, 1), overlap=4, steps=40, cfl=0.05,
                           precision="fp32"),
              W.small_case(3, 15, parts=(1, 2, 2), overlap=3, steps=50, cfl=0.05,
                           precision="fp32")]
    probs[2] = probs[2].replace(max_steps=10 ** 6, tol=5e-3)   # one stops early
    return probs


@pytest.mark.parametrize("graphs", [1, 0])
def test_one_or_two_groups_give_the_same_bits(graphs):
    probs = _batch()
    one = pma.solve_many(probs, groups=1, use_graphs=graphs, window_steps=16)
    two = pma.solve_many(probs, groups=2, use_graphs=graphs, window_steps=16)
    for (a, _, ia), (b, _, ib) in zip(one, two):
        np.testing.assert_array_equal(a, b)
        assert ia.steps == ib.steps and ia.status == ib.status


def test_group_timing_counts_steps():
    probs = _batch()
    with pma.Context(window_steps=16, time_sweeps=4, groups=2) as ctx:
        ids = [ctx.submit(p) for p in probs]
        ctx.run()
        _, s = pma.pma_get_stats(ctx.h, 0)
        for p, i in zip(probs, ids):
            ctx.mesh(p, i)
    assert s.sweep_kernel_launches > 0 and s.sweep_kernel_ms > 0
    assert s.sweep_steps >= s.sweep_kernel_launches
    # two groups per class with work: two sweep launches per (step, class)
    assert s.sweep_launches > s.sweep_steps
    with pytest.raises(pma.PmaError):
        pma.Context(groups=3)
