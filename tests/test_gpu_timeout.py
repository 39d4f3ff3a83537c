"""The bounded device waits: a look-back partition that never publishes (the
test-stall flag, test use only) makes the partitions behind it give up after
their short limit, record AGS_ERR_TIMEOUT with the stage in the detail word,
and finish -- the kernel returns, the context stays usable, and nothing is
written outside the buffers.  No GPU fault is involved: the wait simply runs
out."""
import numpy as np
import pytest
import torch

from paper_2604_18980_gb300 import binding as B
from paper_2604_18980_gb300 import render as R
from paper_2604_18980_gb300 import synth

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

STAGE_EMIT, STAGE_SORT = 1, 2
GUARD = 4096


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2604_18980_gb300 import build
    build.build()
    B.lib()


def _renderer():
    scene, cams, _ = synth.workload("c1_cube16k_256", n=16384, width=256, height=256)
    r = R.Renderer(R.scene_to_device(scene), cams, B.AGS_SCALE_PLAIN, presort=False)
    r.forward()
    r.check()
    return r


def test_emission_look_back_gives_up_and_reports():
    r = _renderer()
    cap = r.capacity
    assert r.n > 4 * 1024          # several look-back partitions behind the stalled one
    keys = torch.full((cap + GUARD,), -7, dtype=torch.int64, device="cuda")
    vals = torch.full((cap + GUARD,), -7, dtype=torch.int32, device="cuda")
    npairs = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.zeros(4, dtype=torch.int64, device="cuda")
    B.ags_emit_pairs(r.proj, r.n, r.cams, keys, vals, cap, npairs, st, r.ws_emit, flags=B.AGS_EMIT_TEST_STALL)
    code, detail = B.ags_check(st, raise_on_error=False)
    assert code == B.AGS_ERR_TIMEOUT and detail == STAGE_EMIT
    assert torch.all(keys[cap:] == -7) and torch.all(vals[cap:] == -7)
    # the context is still usable: the same call without the stall gives the real pairs
    st.zero_()
    B.ags_emit_pairs(r.proj, r.n, r.cams, keys, vals, cap, npairs, st, r.ws_emit)
    B.ags_check(st)
    assert int(npairs.item()) == r.pairs()


@pytest.mark.parametrize("extra,count", [(0, 50000), (B.AGS_SORT_PERSISTENT, 50000),
                                         (B.AGS_SORT_PERSISTENT, 4000000)])
def test_sort_look_back_gives_up_and_reports(extra, count):
    """13 partitions of 4096 keys, and (persistent passes) about 980, more than
    the blocks resident at once, so that blocks go on to further partitions
    after the one that gave up."""
    rng = np.random.default_rng(2)
    keys = rng.integers(0, 1 << 20, count).astype(np.uint32)
    k = torch.zeros(count + GUARD, dtype=torch.int32, device="cuda")
    k[:count] = torch.from_numpy(keys.view(np.int32))
    v = torch.arange(count + GUARD, dtype=torch.int32, device="cuda")
    ka = torch.full_like(k, -7)
    va = torch.full_like(v, -7)
    n = torch.tensor([count], dtype=torch.int64, device="cuda")
    st = torch.zeros(4, dtype=torch.int64, device="cuda")
    ws = torch.empty(B.ags_sort_workspace_bytes(count), dtype=torch.uint8, device="cuda")
    alt = B.ags_sort32(k, v, ka, va, n, count, 0, 20, 7, None, 0, st, ws,
                       flags=B.AGS_SORT_TEST_STALL | extra)
    code, detail = B.ags_check(st, raise_on_error=False)
    assert code == B.AGS_ERR_TIMEOUT and detail == STAGE_SORT
    assert torch.all(ka[count:] == -7) and torch.all(va[count:] == -7)
    assert torch.all(k[count:] == 0) and torch.all(v[count:] == torch.arange(count, count + GUARD, device="cuda",
                                                                              dtype=torch.int32))
    # usable afterwards: a clean sort of the same keys is the stable order
    k[:count] = torch.from_numpy(keys.view(np.int32))
    v[:count] = torch.arange(count, dtype=torch.int32, device="cuda")
    st.zero_()
    alt = B.ags_sort32(k, v, ka, va, n, count, 0, 20, 7, None, 0, st, ws, flags=extra)
    B.ags_check(st)
    out = (va if alt else v)[:count].cpu().numpy()
    np.testing.assert_array_equal(out, np.argsort(keys, kind="stable"))
