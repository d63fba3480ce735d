"""The autotuner measures every compiled work shape and window length on a
scratch context and returns the fastest; the tuned options solve the batch
within the parity tolerances of the oracle."""
import numpy as np
import pytest

import oracle
from paper_2006_14602_gb300 import pma
from paper_2006_14602_gb300 import workloads as W
from paper_2006_14602_gb300.autotune import autotune

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    from paper_2006_14602_gb300 import build
    build.build()
    pma.load()


def test_autotune_picks_a_measured_candidate():
    probs = W.config4(seed=9, count=24, max_steps=100, size_range=(17, 120))
    probs += [W.small_case(3, 21, parts=(2, 1, 2), overlap=4, steps=60, precision="fp32")]
    best = autotune(probs, windows=2, window_candidates=(16, 32), trial_steps=16)
    rates = best["rates"]
    assert all(v > 0 for v in rates.values())
    assert "tile_2d=%d" % best["tile_2d"] in rates and "tile_3d=%d" % best["tile_3d"] in rates
    assert rates["tile_2d=%d" % best["tile_2d"]] == max(v for k, v in rates.items()
                                                         if k.startswith("tile_2d"))
    assert best["window_steps"] in (16, 32)
    # the batch itself is untouched and solves with the tuned options
    p = probs[3].replace(precision="fp32")
    ref = oracle.solve(p.replace(precision="fp64"))
    x, _, info = pma.solve(p, want_psi=False, tile_2d=best["tile_2d"],
                           window_steps=best["window_steps"])
    assert info.steps == ref.steps
    assert np.abs(x - ref.x).max() <= 1e-5
