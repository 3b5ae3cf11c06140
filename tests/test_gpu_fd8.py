"""GPU parity of the 8th-order finite-difference option (Sec. III.C: 9-point
centred first and second derivatives, 4 ghost cells per box, Kreiss-Oliger
dissipation still r = 4) against the CPU oracle on the same seeded inputs:
the wave tolerance 1e-12 and the Z4c tolerance 1e-10 of the 4th-order path."""
import numpy as np
import pytest

from helpers import fetch, init_arrays, load, make_oracle, max_rel_diff
from paper_2503_09629_gb300 import workloads as W

pytestmark = pytest.mark.gpu

WAVE_TOL = 1e-12
Z4C_TOL = 1e-10


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
    assert ctx.ghost == 4
    o = make_oracle(orc, h)
    load(ctx, h, arrays)
    load(o, h, arrays)
    ctx.sc_advance(nsteps)
    o.advance(nsteps)
    err = max_rel_diff(fetch(ctx, h), fetch(o, h))
    assert abs(ctx.sc_get_time() - o.time) < 1e-15
    ctx.close()
    return err


def test_standing_wave_2level_32_fd8(sc, orc):
    h = W.standing_wave_2level(32)
    h.fd_order = 8
    err = _parity(sc, orc, h, 32)
    assert err <= WAVE_TOL, err


def test_gaussian_3level_uneven_boxes_fd8(sc, orc):
    h = W.gaussian_3level(64, 1)
    h.fd_order = 8
    err = _parity(sc, orc, h, 8, noise_seed=1)
    assert err <= WAVE_TOL, err


def test_ragged_boxes_fd8(sc, orc):
    h = W.Hierarchy(system=W.WAVE,
                    boxes=[W.split_uniform(W.cube(0, 24), (3, 1, 2)),
                           [((12, 12, 12), (33, 21, 35)), ((12, 22, 12), (33, 35, 35))]],
                    ncells0=(24, 24, 24), origin=(0.0, 0.0, 0.0), h0=1.0 / 24,
                    id_kind=W.ID_STANDING_WAVE, id_params=[1.0, 1.0, 2.0, 1.0], fd_order=8)
    err = _parity(sc, orc, h, 6)
    assert err <= WAVE_TOL, err


def test_bl_3level_16_coarse_steps_fd8(sc, orc):
    h = W.bl_3level(20)
    h.fd_order = 8
    err = _parity(sc, orc, h, 16)
    assert err <= Z4C_TOL, err


def test_constraints_fd8(sc, orc):
    h = W.bl_3level(20)
    h.fd_order = 8
    arrays = init_arrays(h)
    ctx = sc.Context(h)
    o = make_oracle(orc, h)
    load(ctx, h, arrays)
    load(o, h, arrays)
    ctx.sc_advance(2)
    o.advance(2)
    for l in range(3):
        g = ctx.sc_get_constraints(l, 0)
        r = o.constraints(l, 0)
        for q in range(7):
            scale = max(np.abs(r[q]).max(), 1e-12)
            assert np.abs(g[q] - r[q]).max() / scale <= 1e-9, (l, q)


def test_fd8_and_fd4_differ_by_truncation_only(sc):
    """Same data, 4th- and 8th-order differences: the runs differ (the
    option is live) by no more than the 4th-order truncation error."""
    out = []
    for order in (4, 8):
        h = W.standing_wave_2level(32)
        h.fd_order = order
        ctx = sc.Context(h)
        ctx.sc_set_initial_data(h.id_kind, h.id_params)
        ctx.sc_advance(8)
        out.append(ctx.sc_get_field(1, 0, 0))
        ctx.close()
    d = np.abs(out[0] - out[1]).max()
    assert 1e-9 < d < 1e-3, d
