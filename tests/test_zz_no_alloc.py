"""The allocation-free forward-sets entry point against the regular one.

ik_forward_sets_noalloc serves callers that cannot allocate GPU memory when
they need an answer (an arena allocator owning the device, a real-time loop
that must not pay cudaMalloc's synchronisation); its scratch is a fixed
device array inside the library.  It must give exactly the sets that
ik_forward_sets gives, call after call, although every call reuses (and
finds the previous call's leftovers in) the same scratch.  This file is named
to run last.
"""
import numpy as np
import pytest

import scenegen as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ik():
    from paper_1906_10678_b300 import build
    build.build()
    from paper_1906_10678_b300 import ik as mod
    return mod


def _case(ik, torch, scene, root):
    """(device occupancy words, sets from ik_forward_sets) for one scene."""
    with ik.Grid(*scene.shape) as g:
        ik.ik_set_boxes(g.h, scene.boxes)
        occ = ik.ik_get_obstacles(g.h)
        want = ik.ik_forward_sets(g.h, scene.lengths, root)
    occ_d = torch.from_numpy(occ.view(np.int32).copy()).cuda()
    return occ_d, want


def test_noalloc_forward_sets_match_regular_entry_point(ik):
    import torch
    torch.cuda.set_device(0)
    cases = [(G.c2_scene(1), (64, 64, 0)), (G.c1_scene(3), (16, 16, 0)),
             (G.c1_scene(5), (10, 20, 3))]
    for scene, root in cases:  # consecutive calls with different arms and grids
        occ_d, want = _case(ik, torch, scene, root)
        S = len(scene.lengths)
        out = torch.full((want.size,), -1, dtype=torch.int32, device="cuda")
        ik.ik_forward_sets_noalloc(occ_d, scene.shape, scene.lengths, root, out)
        got = out.cpu().numpy().view(np.uint32).reshape(S + 1, -1)
        assert (got == want).all(), scene.name
    # the same first case again, after the scratch held the other arms; this
    # call must not change the device's free memory or torch's allocations
    scene, root = cases[0]
    occ_d, want = _case(ik, torch, scene, root)
    out = torch.zeros((want.size,), dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    ik.ik_forward_sets_noalloc(occ_d, scene.shape, scene.lengths, root, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0 and torch.cuda.memory_allocated() == alloc0
    assert (out.cpu().numpy().view(np.uint32).reshape(len(scene.lengths) + 1, -1) == want).all()


def test_noalloc_rejects_arms_beyond_its_scratch(ik):
    import torch
    occ = torch.zeros(4 * 32 * 32, dtype=torch.int32, device="cuda")
    out = torch.zeros(9 * 4 * 32 * 32, dtype=torch.int32, device="cuda")
    with pytest.raises(ik.IkError) as err:
        ik.ik_forward_sets_noalloc(occ, (128, 32, 32), [30] * 8, (1, 1, 1), out)
    assert err.value.code == ik.IK_ERR_UNSUPPORTED
