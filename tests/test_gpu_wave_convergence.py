"""Fourth-order self-convergence of the GPU path on the 3-level scalar-wave
workload (seeded uneven boxes; Gaussian pulse of width 0.05 plus 1e-3 of
smooth seeded noise): the same physical box layout at 64^3, 128^3 and 256^3
base resolution (the seeded layout scaled by 2 and 4), evolved to the same
time with subcycling (Sec. II) and dense-output ghost filling.  The finest
level of each run is mapped to the cell centres of the next coarser run by
6-point Lagrange interpolation at the midpoint (6th-order accurate), and
order = log2(|u64 - I u128| / |u128 - I u256|) must be 4 within 0.3 (the
paper's Fig. 2 shows 4th-order convergence of the wave with subcycling)."""
import numpy as np
import pytest

from paper_2503_09629_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MID6 = np.array([3.0, -25.0, 150.0, 150.0, -25.0, 3.0]) / 256.0  # Lagrange weights at the midpoint


@pytest.fixture(scope="module")
def sc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_09629_gb300 as m
    m.build()
    return m


def _finest(ctx, h):
    boxes = h.boxes[2]
    lo = np.min([b[0] for b in boxes], axis=0)
    hi = np.max([b[1] for b in boxes], axis=0)
    out = np.full(tuple((hi - lo + 1)[::-1]), np.nan)
    for bi, (blo, bhi) in enumerate(boxes):
        out[tuple(slice(blo[d] - lo[d], bhi[d] - lo[d] + 1) for d in (2, 1, 0))] = ctx.sc_get_field(2, bi, 0)
    return out


def _to_coarse(u):
    for ax in range(3):
        n = u.shape[ax] // 2
        u = np.stack([np.tensordot(np.take(u, np.arange(2 * C - 2, 2 * C + 4), axis=ax), MID6, axes=([ax], [0]))
                      for C in range(2, n - 2)], axis=ax)
    return u


def test_wave_3level_self_convergence_order_four(sc):
    fine = {}
    for n in (64, 128, 256):
        h = W.gaussian_3level(n, 0)
        ctx = sc.Context(h)
        for l in range(h.nlevels):
            for b in range(len(h.boxes[l])):
                a = W.initial_fields(h, l, b, noise_seed=0)
                for f in range(2):
                    ctx.sc_set_field(l, b, f, a[f])
        ctx.sc_advance(32 * n // 64)
        fine[n] = _finest(ctx, h)
        ctx.close()
    assert not np.isnan(fine[64]).any()  # the level-2 boxes tile their bounding box
    e1 = np.abs(fine[64][2:-2, 2:-2, 2:-2] - _to_coarse(fine[128])).max()
    e2 = np.abs(fine[128][2:-2, 2:-2, 2:-2] - _to_coarse(fine[256])).max()
    order = np.log2(e1 / e2)
    assert abs(order - 4.0) < 0.3, (e1, e2, order)
