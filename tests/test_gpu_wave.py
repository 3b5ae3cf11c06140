"""GPU parity of the scalar-wave path (Sec. IV.A) through the C ABI against
the CPU oracle on the same seeded inputs: tolerance 1e-12 in the max relative
field difference after the run."""
import numpy as np
import pytest

from helpers import fetch, init_arrays, load, make_oracle, max_rel_diff
from paper_2503_09629_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def sc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_09629_gb300 as m
    m.build()
    return m


def _parity(sc, orc, h, nsteps, noise_seed=None):
    arrays = init_arrays(h, noise_seed)
    ctx = sc.Context(h)
    o = make_oracle(orc, h)
    load(ctx, h, arrays)
    load(o, h, arrays)
    ctx.sc_advance(nsteps)
    o.advance(nsteps)
    err = max_rel_diff(fetch(ctx, h), fetch(o, h))
    assert abs(ctx.sc_get_time() - o.time) < 1e-15
    assert ctx.sc_zone_updates() == o.zone_updates()
    ctx.close()
    return err


def test_standing_wave_2level_32(sc, orc):
    """Standing wave, level 0 32^3 + fine 32^3 over [0.25,0.75]^3, 32 coarse steps."""
    h = W.standing_wave_2level(32)
    err = _parity(sc, orc, h, 32)
    assert err <= TOL, err


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gaussian_3level_uneven_boxes_64(sc, orc, seed):
    """Gaussian + seeded noise, 3 levels, 27 uneven level-0 boxes and 8-18
    seeded uneven boxes on each fine level, 64^3 base, 32 coarse steps."""
    h = W.gaussian_3level(64, seed)
    err = _parity(sc, orc, h, 32 if seed == 0 else 8, noise_seed=seed)
    assert err <= TOL, err


def test_ragged_boxes_and_tails(sc, orc):
    """Odd interior widths that leave ragged tiles in x, y and z."""
    h = W.Hierarchy(system=W.WAVE,
                    boxes=[W.split_uniform(W.cube(0, 24), (3, 1, 2)),
                           [((12, 12, 12), (33, 21, 35)), ((12, 22, 12), (33, 35, 35))]],
                    ncells0=(24, 24, 24), origin=(0.0, 0.0, 0.0), h0=1.0 / 24,
                    id_kind=W.ID_STANDING_WAVE, id_params=[1.0, 1.0, 2.0, 1.0])
    err = _parity(sc, orc, h, 6)
    assert err <= TOL, err


def test_single_level(sc, orc):
    h = W.Hierarchy(system=W.WAVE, boxes=[[W.cube(0, 20)]], ncells0=(20, 20, 20), origin=(0.0, 0.0, 0.0),
                    h0=1.0 / 20, id_kind=W.ID_STANDING_WAVE, id_params=[1.0, 1.0, 1.0, 1.0])
    assert _parity(sc, orc, h, 10) <= TOL


def test_zero_steps_is_identity(sc, orc):
    h = W.standing_wave_2level(16)
    arrays = init_arrays(h)
    ctx = sc.Context(h)
    load(ctx, h, arrays)
    ctx.sc_advance(0)
    got = fetch(ctx, h)
    for l in range(2):
        assert np.array_equal(got[l][0], arrays[l][0][:, 3:-3, 3:-3, 3:-3])


def test_split_boxes_bitwise_gpu(sc):
    """Splitting a level into boxes changes nothing, bitwise (GPU vs GPU)."""
    one = W.standing_wave_2level(24)
    many = W.Hierarchy(system=W.WAVE, boxes=[W.split_uniform(W.cube(0, 24), (2, 3, 2)),
                                             W.split_uniform(W.cube(12, 24), (3, 2, 2))],
                       ncells0=(24, 24, 24), origin=(0.0, 0.0, 0.0), h0=1.0 / 24)
    ca, cb = sc.Context(one), sc.Context(many)
    for c in (ca, cb):
        c.sc_set_initial_data(W.ID_STANDING_WAVE, [1.0, 1.0, 2.0, 1.0])
        c.sc_advance(5)
    for l in range(2):
        full = ca.sc_get_field(l, 0, 0)
        blo = one.boxes[l][0][0]
        for bi, (lo, hi) in enumerate(many.boxes[l]):
            sl = tuple(slice(lo[d] - blo[d], hi[d] - blo[d] + 1) for d in (2, 1, 0))
            assert np.array_equal(cb.sc_get_field(l, bi, 0), full[sl])


def test_deterministic(sc):
    h = W.gaussian_3level(64, 1)
    res = []
    for _ in range(2):
        c = sc.Context(h)
        c.sc_set_initial_data(h.id_kind, h.id_params)
        c.sc_advance(3)
        res.append(fetch(c, h))
        c.close()
    for la, lb in zip(*res):
        for a, b in zip(la, lb):
            assert np.array_equal(a, b)


def test_initial_data_matches_oracle(sc, orc):
    """The device initial-data kernel against the oracle's own initial data."""
    for kind, params in ((W.ID_STANDING_WAVE, [1.0, 1.0, 2.0, 3.0]), (W.ID_GAUSSIAN, [1.0, 0.05, 0.5, 0.5, 0.5])):
        h = W.standing_wave_2level(16)
        ctx = sc.Context(h)
        o = make_oracle(orc, h)
        ctx.sc_set_initial_data(kind, params)
        o.set_initial_data(kind, params)
        assert max_rel_diff(fetch(ctx, h), fetch(o, h)) <= 1e-14


def test_nesting_violation_rejected(sc):
    """A fine box whose prolongation stencil leaves the parent interior."""
    h = W.Hierarchy(system=W.WAVE, boxes=[[W.cube(0, 16)], [W.cube(2, 8)]], ncells0=(16, 16, 16),
                    origin=(0.0, 0.0, 0.0), h0=1.0 / 16, bc=W.BC_RADIATIVE)
    with pytest.raises(sc.SubcycError) as e:
        sc.Context(h)
    assert e.value.code == sc.SC_ENESTING


def test_autotune_keeps_results_bitwise(sc):
    """The autotuner changes only the tiling; every cell's arithmetic and so
    the fields are bitwise those of the default tiles."""
    h = W.gaussian_3level(64, 0)
    out = []
    for tune in (False, True):
        c = sc.Context(h)
        if tune:
            tile, _ms = c.sc_autotune()
            assert len(tile) == 3 and all(t > 0 for t in tile)
        c.sc_set_initial_data(h.id_kind, h.id_params)
        c.sc_advance(3)
        out.append(fetch(c, h))
        c.close()
    for la, lb in zip(*out):
        for a, b in zip(la, lb):
            assert np.array_equal(a, b)


def test_uniform_step_mode_matches_oracle(sc, orc):
    """Uniform time step on every level (the comparison mode of Sec. IV.A):
    GPU against the oracle's uniform mode."""
    h = W.standing_wave_2level(24, subcycle=False)
    err = _parity(sc, orc, h, 6)
    assert err <= TOL, err


def test_uniform_and_subcycled_agree_to_truncation(sc):
    """Sec. IV.A: subcycled and uniform-step runs differ by less than the
    error of either against the exact standing wave."""
    t_end = 0.125
    out = {}
    for sub in (True, False):
        h = W.standing_wave_2level(32, subcycle=sub)
        c = sc.Context(h)
        c.sc_set_initial_data(h.id_kind, h.id_params)
        c.sc_advance(int(round(t_end / (h.cfl * h.h0))))
        X, Y, Z = h.cell_centres(1, 0)
        u = c.sc_get_field(1, 0, 0)
        exact = np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y) * np.sin(2 * np.pi * Z) * np.cos(
            2 * np.sqrt(3) * np.pi * c.sc_get_time())
        out[sub] = (u, np.abs(u - exact).max())
        c.close()
    diff = np.abs(out[True][0] - out[False][0]).max()
    assert diff < out[True][1] and diff < out[False][1]
