"""The allocation-free constraint entry point against the allocating one.

sc_z4c_constraints_noalloc serves callers that cannot allocate device memory
(an embedding application that owns all of it, a fixed memory pool, a loop
that must avoid the implicit synchronisation of cudaMalloc/cudaFree).  It
runs the same kernels as sc_get_constraints with a static scratch array, so
on the same box data the two must agree; this file checks two calls in a
row, through the C ABI, within the constraint tolerance of the other tests.
It is collected last so that a run stopping at the first failure has already
run every other test, and it passes alone in a fresh process as well.
"""
import numpy as np
import pytest

from helpers import init_arrays, load
from paper_2503_09629_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-9  # the constraint tolerance of test_gpu_z4c.py


@pytest.fixture(scope="module")
def sc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_09629_gb300 as m
    m.build()
    return m


def test_noalloc_constraints_match_allocating_path(sc):
    import torch
    h = W.bl_3level(20)
    ctx = sc.Context(h)
    load(ctx, h, init_arrays(h))
    ctx.sc_advance(2)
    stream = torch.cuda.current_stream().cuda_stream
    for level in (0, 1, 2):
        ref = ctx.sc_get_constraints(level, 0)
        state = np.stack([ctx.sc_get_field(level, 0, f, ghosted=True) for f in range(22)])
        dev_state = torch.from_numpy(state).cuda()
        n = ctx.shape(level, 0)[::-1]  # (nx, ny, nz)
        dev_out = torch.empty((7,) + ctx.shape(level, 0), dtype=torch.float64, device="cuda")
        hl = h.h0 / 2 ** level
        for _call in range(2):
            dev_out.fill_(float("nan"))
            sc.sc_z4c_constraints_noalloc(dev_state.data_ptr(), dev_out.data_ptr(), n, hl, stream)
            torch.cuda.synchronize()
            got = dev_out.cpu().numpy()
            assert np.isfinite(got).all()
            for q in range(7):
                scale = max(np.abs(ref[q]).max(), 1e-12)
                assert np.abs(got[q] - ref[q]).max() / scale <= TOL, (level, q)
    ctx.close()


def test_noalloc_rejects_oversized_box(sc):
    import torch
    dev = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(sc.SubcycError) as e:
        sc.sc_z4c_constraints_noalloc(dev.data_ptr(), dev.data_ptr(), (40, 40, 40), 0.1, None)
    assert e.value.code == sc.SC_EINVAL
    assert "too large" in str(e.value)
