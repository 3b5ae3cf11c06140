"""The allocation-free constraint entry point against the allocating one.

sc_z4c_constraints_noalloc serves callers that cannot allocate device memory
(an embedding application that owns all of it, a fixed memory pool, a loop
that must avoid the implicit synchronisation of cudaMalloc/cudaFree).  It
runs the same derivative and constraint kernels as sc_get_constraints of a
4th-order context, with the same tile shape, on the same ghosted box data,
so the two must agree bit for bit: an indexing or stride slip in the dense
box layout would otherwise hide inside a tolerance.  This file checks two
calls in a row through the C ABI, on the legacy stream and on a non-default
stream.  It is collected last so that a run stopping at the first failure has
already run every other test, and it passes alone in a fresh process as well.
"""
import numpy as np
import pytest

from helpers import init_arrays, load
from paper_2503_09629_gb300 import workloads as W

pytestmark = pytest.mark.gpu


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
    side = torch.cuda.Stream()
    for level in (0, 1, 2):
        ref = ctx.sc_get_constraints(level, 0)
        state = np.stack([ctx.sc_get_field(level, 0, f, ghosted=True) for f in range(22)])
        dev_state = torch.from_numpy(state).cuda()
        n = ctx.shape(level, 0)[::-1]  # (nx, ny, nz)
        dev_out = torch.empty((7,) + ctx.shape(level, 0), dtype=torch.float64, device="cuda")
        hl = h.h0 / 2 ** level
        torch.cuda.synchronize()
        for stream in (None, side):
            for _call in range(2):
                with torch.cuda.stream(stream if stream is not None else torch.cuda.default_stream()):
                    dev_out.fill_(float("nan"))
                    sc.sc_z4c_constraints_noalloc(dev_state.data_ptr(), dev_out.data_ptr(), n, hl,
                                                  stream.cuda_stream if stream is not None else None)
                torch.cuda.synchronize()
                got = dev_out.cpu().numpy()
                assert np.isfinite(got).all()
                assert np.array_equal(got, ref), (level, stream, np.abs(got - ref).max())
    ctx.close()


def test_noalloc_rejects_oversized_box(sc):
    import torch
    dev = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(sc.SubcycError) as e:
        sc.sc_z4c_constraints_noalloc(dev.data_ptr(), dev.data_ptr(), (40, 40, 40), 0.1, None)
    assert e.value.code == sc.SC_EINVAL
    assert "too large" in str(e.value)
