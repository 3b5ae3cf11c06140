"""GPU parity of RK2 (explicit midpoint) and RK3 (Heun's third-order method)
subcycling -- the extension Sec. V of the paper leaves to future work --
against the CPU oracle on the same seeded inputs: wave 1e-12, Z4c 1e-10."""
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


@pytest.mark.parametrize("rk", [2, 3])
def test_standing_wave_2level_32(sc, orc, rk):
    """RK3: 32 coarse steps.  RK2 (midpoint) grows the highest wave modes by
    |R(i z)| = (1 + z^4 / 4)^(1/2) = 1.118 per fine step at CFL 0.25 (z = 1), so
    rounding differences between the two sides grow about 1260x over 64 fine
    steps; it runs 8 coarse steps (16 fine, growth at most 6) at the same
    tolerance."""
    h = W.standing_wave_2level(32)
    h.rk_order = rk
    assert _parity(sc, orc, h, 32 if rk == 3 else 8) <= WAVE_TOL


@pytest.mark.parametrize("rk", [2, 3])
def test_gaussian_3level_uneven_boxes(sc, orc, rk):
    h = W.gaussian_3level(64, 0)
    h.rk_order = rk
    assert _parity(sc, orc, h, 8 if rk == 3 else 4, noise_seed=0) <= WAVE_TOL


@pytest.mark.parametrize("rk", [2, 3])
def test_bl_3level_z4c(sc, orc, rk):
    h = W.bl_3level(20)
    h.rk_order = rk
    assert _parity(sc, orc, h, 16 if rk == 3 else 8) <= Z4C_TOL


def test_rk3_with_8th_order_differences(sc, orc):
    h = W.bl_3level(20)
    h.rk_order = 3
    h.fd_order = 8
    assert _parity(sc, orc, h, 4) <= Z4C_TOL


@pytest.mark.parametrize("rk", [2, 3])
def test_uniform_step_mode(sc, orc, rk):
    h = W.standing_wave_2level(32, subcycle=False)
    h.rk_order = rk
    assert _parity(sc, orc, h, 4) <= WAVE_TOL


def test_rk3_k4_is_f_of_new_state_and_unused_vectors_rejected(sc):
    """RK3: the level with a finer level keeps k4 = f(y_{n+1}) (for a standing
    wave, its Pi component is the Laplacian of the new u); the finest level
    has no k4 and the call is rejected.  RK2 has no k3."""
    h = W.standing_wave_2level(16)
    h.rk_order = 3
    ctx = sc.Context(h)
    ctx.sc_set_initial_data(h.id_kind, h.id_params)
    ctx.sc_advance(1)
    k3 = ctx.sc_debug_get_vector(1, 0, 6, 0)
    assert np.isfinite(k3).all() and np.abs(k3).max() > 0
    k4_u = ctx.sc_debug_get_vector(0, 0, 7, 0)
    pi_new = ctx.sc_debug_get_vector(0, 0, 0, 1)
    # d_t u = Pi: k4's u component is the Pi of the level's new state, except
    # where restriction from the fine box (cells 4..11 of 16) replaced it
    covered = np.zeros_like(pi_new, dtype=bool)
    covered[4:12, 4:12, 4:12] = True
    assert np.array_equal(k4_u[~covered], pi_new[~covered])
    assert np.isfinite(k4_u).all()
    with pytest.raises(Exception):
        ctx.sc_debug_get_vector(1, 0, 7, 0)
    ctx.close()
    h.rk_order = 2
    ctx = sc.Context(h)
    with pytest.raises(Exception):
        ctx.sc_debug_get_vector(0, 0, 6, 0)
    ctx.close()
