"""Host-buffer delivery of meshes through the C ABI: pma_get_mesh_batch
packs the meshes of several finished requests into one caller-owned host
buffer; it must equal pma_get_mesh request by request (bitwise: the same
combination kernel), release the requests, and reject bad id lists without
releasing anything."""
import ctypes as C

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
    probs = W.config4(count=9, max_steps=60, size_range=(17, 129))
    probs.append(W.small_case(3, 13, parts=(2, 1, 2), overlap=3, steps=30, cfl=0.05,
                              precision="fp32"))
    return probs


@pytest.mark.parametrize("pinned", [True, False])
def test_batch_host_delivery_equals_single_requests(pinned):
    import torch
    probs = _batch()
    with pma.Context() as ctx:
        ids = [ctx.submit(p) for p in probs]
        ctx.run()
        singles = [ctx.mesh(p, i)[0] for p, i in zip(probs, ids)]
    sizes = [p.dim * p.nodes for p in probs]
    host = torch.empty(sum(sizes), dtype=torch.float64, pin_memory=pinned)
    host.fill_(float("nan"))
    infos = (pma.pma_info * len(probs))()
    with pma.Context() as ctx:
        ids = [ctx.submit(p) for p in probs]
        ctx.run()
        st = pma.pma_get_mesh_batch(ctx.h, ids, host.data_ptr(), infos)
        assert st == pma.PMA_OK, pma.pma_last_error()
        # released: the ids are gone
        assert pma.pma_get_info(ctx.h, ids[0])[0] == pma.PMA_ERR_NOT_FOUND
        _, counts = pma.pma_counts(ctx.h)
        assert counts == (0, 0, 0)
    flat = host.numpy()
    off = 0
    for p, x, n, info in zip(probs, singles, sizes, infos):
        np.testing.assert_array_equal(flat[off:off + n], x.ravel())
        assert info.steps == p.max_steps
        off += n


def test_batch_host_delivery_rejects_bad_lists():
    import torch
    probs = _batch()[:3]
    host = torch.empty(sum(p.dim * p.nodes for p in probs), dtype=torch.float64)
    with pma.Context() as ctx:
        ids = [ctx.submit(p) for p in probs]
        ctx.run()
        assert pma.pma_get_mesh_batch(ctx.h, [ids[0], ids[0]], host.data_ptr()) == \
            pma.PMA_ERR_INVALID
        assert pma.pma_get_mesh_batch(ctx.h, [ids[0], 987654], host.data_ptr()) == \
            pma.PMA_ERR_NOT_FOUND
        assert pma.pma_get_mesh_batch(ctx.h, ids, 0) == pma.PMA_ERR_INVALID
        # nothing was released by the failed calls
        assert pma.pma_counts(ctx.h)[1] == (0, 0, 3)
        assert pma.pma_get_mesh_batch(ctx.h, ids, host.data_ptr()) == pma.PMA_OK
        pending = ctx.submit(probs[0].replace(max_steps=10 ** 6))
        assert pma.pma_get_mesh_batch(ctx.h, [pending], host.data_ptr()) == pma.PMA_ERR_BUSY
