"""Autotuner of the batched path: work shapes and steps per graph window.

The sweep kernels are compiled for a few work shapes (2D: threads x band
nodes; 3D: threads x box nodes per plane x planes) and advance the batch in
CUDA-graph windows of `window_steps` steps.  Which shape and window length
are fastest depends on the batch: how many subdomain nodes a step holds,
how ragged the subdomains are, 2D or 3D, FP32 or FP64.  `autotune` measures
instead of guessing: it submits the same requests to a scratch context,
runs a few windows per candidate and keeps the candidate with the most
node-updates per second of device time (the library's CUDA-event timing of
the stepping windows).  The scratch context is destroyed afterwards; the
caller's requests are untouched.

A shape changes the order in which theta's partial sums are added, so
results under different shapes agree to rounding (the parity tolerances),
not bitwise; a context keeps one shape per kernel class for its lifetime.
"""
from typing import Dict, Optional, Sequence

from . import pma


def _count(option: str) -> int:
    """Number of compiled shapes for a tile option (ids 0..n-1)."""
    n = 0
    with pma.Context(0) as ctx:
        while True:
            try:
                ctx.set(option, n)
            except pma.PmaError:
                return n
            n += 1


def _rate(probs, steps: int, windows: int, device: int, **options) -> float:
    """Node-updates per second of window device time, after one warm-up
    window, for `probs` capped at enough steps to stay busy."""
    trial = [p.replace(max_steps=steps * (windows + 2), tol=0.0) for p in probs]
    with pma.Context(device, window_steps=steps, **options) as ctx:
        for p in trial:
            ctx.submit(p)
        st = pma.pma_admit(ctx.h)
        if st != pma.PMA_OK:
            raise pma.PmaError("pma_admit", st)
        ctx.run(1)
        pma.pma_get_stats(ctx.h, 1)
        ctx.run(windows)
        _, s = pma.pma_get_stats(ctx.h, 0)
    return s.node_updates / (s.window_ms / 1e3) if s.window_ms > 0 else 0.0


def autotune(probs: Sequence, device: int = 0, windows: int = 3,
             window_candidates: Sequence[int] = (32, 64, 128, 256),
             trial_steps: int = 32, **options) -> Dict:
    """Pick tile_2d, tile_3d and window_steps for the batch `probs`.

    Shapes are tried first (at `trial_steps` steps per window), the 2D shape
    with the default 3D shape and then the 3D shape with the chosen 2D one,
    each only if the batch holds requests of that dimension; then the window
    lengths with the chosen shapes.  Returns the choice and the measured
    rates (node-updates/s) of every candidate."""
    dims = {p.dim for p in probs}
    best = {"tile_2d": 0, "tile_3d": 0, "window_steps": trial_steps}
    rates: Dict[str, float] = {}
    for dim, opt in ((2, "tile_2d"), (3, "tile_3d")):
        if dim not in dims:
            continue
        scores = {}
        for t in range(_count(opt)):
            cfg = dict(options, **{k: v for k, v in best.items() if k != "window_steps"})
            cfg[opt] = t
            scores[t] = _rate(probs, trial_steps, windows, device, **cfg)
            rates["%s=%d" % (opt, t)] = scores[t]
        best[opt] = max(scores, key=scores.get)
    wscores = {}
    for w in window_candidates:
        cfg = dict(options, tile_2d=best["tile_2d"], tile_3d=best["tile_3d"])
        wscores[w] = _rate(probs, w, max(1, windows * trial_steps // w), device, **cfg)
        rates["window_steps=%d" % w] = wscores[w]
    best["window_steps"] = max(wscores, key=wscores.get)
    best["rates"] = rates
    return best
