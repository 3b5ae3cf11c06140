"""Moving boxes (puncture-tracking box stacks): regrid and point interpolation on the
GPU against the CPU oracle, and puncture tracking."""
import numpy as np
import pytest

from helpers import fetch, init_arrays, load, make_oracle, max_rel_diff
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


def test_interpolate_matches_oracle(sc, orc):
    h, pos, radii, fm = W.moving_bl(32)
    ctx = sc.Context(h)
    o = make_oracle(orc, h)
    arrays = init_arrays(h)
    load(ctx, h, arrays)
    load(o, h, arrays)
    ctx.sc_advance(1)
    o.advance(1)
    pts = np.random.default_rng(3).uniform(-6, 6, size=(16, 3))
    for f in (0, 18, 19):
        g = ctx.sc_interpolate(pts, f)
        r = o.interpolate(pts, f)
        assert np.abs(g - r).max() <= 1e-10 * max(np.abs(r).max(), 1e-12)


def test_regrid_every_step_matches_oracle(sc, orc):
    """Prescribed puncture motion (so both sides make identical box
    decisions): regrid before each of 4 coarse steps, then compare."""
    h, pos, radii, fm = W.moving_bl(32)
    ctx = sc.Context(h)
    o = make_oracle(orc, h)
    arrays = init_arrays(h)
    load(ctx, h, arrays)
    load(o, h, arrays)
    for step in range(4):
        pos = [(p[0] + (0.15 if p[0] < 0 else -0.15), p[1] + 0.05, p[2]) for p in pos]
        layout = W.moving_layout(h, pos, radii, fm)
        ctx.sc_regrid(layout)
        o.regrid(layout)
        h = W.Hierarchy(**{**h.__dict__, "boxes": layout})
        ctx.sc_advance(1)
        o.advance(1)
    assert max_rel_diff(fetch(ctx, h), fetch(o, h)) <= 1e-10


def test_regrid_same_layout_is_identity_gpu(sc):
    h, pos, radii, fm = W.moving_bl(32)
    ctx = sc.Context(h)
    ctx.sc_set_initial_data(h.id_kind, h.id_params)
    ctx.sc_advance(1)
    before = fetch(ctx, h)
    ctx.sc_regrid(h.boxes)
    for la, lb in zip(before, fetch(ctx, h)):
        for a, b in zip(la, lb):
            assert np.array_equal(a, b)


def test_puncture_tracking_moves_box_stacks(sc):
    """Shift-driven tracking: the punctures of a head-on pair fall inward,
    the finest box stacks follow and stay nested; a regrid that breaks
    nesting is refused and leaves the context usable."""
    h, pos, radii, fm = W.moving_bl(32)
    ctx = sc.Context(h)
    ctx.sc_set_initial_data(h.id_kind, h.id_params)
    dt0 = h.cfl * h.h0
    for _ in range(6):
        pos = W.track_punctures(ctx, pos, dt0)
        ctx.sc_regrid(W.moving_layout(ctx.h, pos, radii, fm))
        ctx.sc_advance(1)
    assert pos[0][0] > -1.5 and pos[1][0] < 1.5
    assert abs(pos[0][0] + pos[1][0]) < 1e-9
    bad = [list(b) for b in ctx.h.boxes]
    bad[3] = [((2, 2, 2), (17, 17, 17))]
    with pytest.raises(sc.SubcycError) as e:
        ctx.sc_regrid(bad)
    assert e.value.code == sc.SC_ENESTING
    ctx.sc_advance(1)
    assert np.isfinite(ctx.sc_get_field(3, 0, 0)).all()
