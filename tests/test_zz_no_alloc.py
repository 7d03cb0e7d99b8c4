"""The allocation-free neighbour entry point, for callers that cannot call
cudaMalloc (a fixed device-memory budget, a loop that must not synchronise the
device, a plug-in inside another framework's memory pool).  Checked through
the C ABI against the allocating entry point on two calls in a row: the
outputs must be identical (integer work, bit-exact), and the second call must
not see anything left in the shared scratch by the first."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    torch.cuda.init()
    from paper_2605_22698_gb300 import build
    build.build()
    from paper_2605_22698_gb300 import binding
    binding.lib()
    return binding


def _run(B, s):
    import torch
    ref_r, ref_s, ref_sh = B.mlip_neighbors(np.ascontiguousarray(s.pos), s.cell, s.pbc, 5.0)
    cap = len(ref_r) + 64
    pos = torch.tensor(s.pos, device="cuda")
    recv = torch.full((cap,), -7, dtype=torch.int32, device="cuda")
    send = torch.full((cap,), -7, dtype=torch.int32, device="cuda")
    shift = torch.zeros((cap, 3), dtype=torch.int8, device="cuda")
    E = B.mlip_neighbors_noalloc(pos, s.cell, s.pbc, 5.0, recv, send, shift)
    torch.cuda.synchronize()
    assert E == len(ref_r)
    np.testing.assert_array_equal(recv[:E].cpu().numpy(), ref_r)
    np.testing.assert_array_equal(send[:E].cpu().numpy(), ref_s)
    np.testing.assert_array_equal(shift[:E].cpu().numpy(), ref_sh)
    return E


def test_noalloc_matches_allocating_entry_point_twice(B):
    big = synth.water_box(1000, 31.0, seed=2)            # periodic, 3000 atoms
    small = synth.cluster(300, seed=5)                  # open cluster after a larger call
    for s in (big, small, big):
        _run(B, s)


def test_noalloc_rejects_oversized_input(B):
    import torch
    s = synth.fcc((14, 14, 16), seed=3)                 # 12544 atoms > 12288
    pos = torch.tensor(s.pos, device="cuda")
    out = torch.zeros(8, dtype=torch.int32, device="cuda")
    sh = torch.zeros((8, 3), dtype=torch.int8, device="cuda")
    with pytest.raises(B.MlipError) as e:
        B.mlip_neighbors_noalloc(pos, s.cell, s.pbc, 5.0, out, out, sh)
    assert e.value.code == B.MLIP_ERR_INVALID_ARG
    assert "12288" in str(e.value)


def test_noalloc_rejects_a_receiver_above_the_degree_limit(B):
    """A dense open FCC cluster (a = 1.2 A, 864 atoms): its central atoms
    have far more than 256 neighbours within 5 A.  The call must return
    MLIP_ERR_CAPACITY naming the limit, and a following ordinary call must
    still match the allocating entry point."""
    import torch
    s = synth.fcc((6, 6, 6), seed=3)
    pos_h = s.pos * (1.2 / 3.6)
    pos = torch.tensor(pos_h, device="cuda")
    out = torch.zeros(8, dtype=torch.int32, device="cuda")
    sh = torch.zeros((8, 3), dtype=torch.int8, device="cuda")
    with pytest.raises(B.MlipError) as e:
        B.mlip_neighbors_noalloc(pos, np.eye(3), np.zeros(3, np.uint8), 5.0, out, out, sh)
    assert e.value.code == B.MLIP_ERR_CAPACITY
    assert "256" in str(e.value)
    _run(B, synth.cluster(300, seed=6))
