"""The persistent coarse-step kernel of the scalar wave (one cooperative
launch per coarse step: every stage of every substep on every level, the
dense-output ghost fills, prolongation and restriction of Sec. II, separated
by grid barriers) against the graph form: the same device-function bodies
compute every value, so the fields must agree bit for bit, for the
benchmark's small wave cases, uneven seeded boxes, the other Runge-Kutta
methods, 8th-order differences and the uniform-step mode."""
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


def _run(sc, h, mode, steps, noise=None):
    ctx = sc.Context(h, exec_mode=mode)
    load(ctx, h, init_arrays(h, noise_seed=noise))
    ctx.sc_advance(steps)
    ctx.sc_synchronize()
    out = fetch(ctx, h), ctx.sc_launches_per_step(), ctx.sc_zone_updates()
    ctx.close()
    return out


def _cases():
    c1 = W.standing_wave_2level(32)
    c2 = W.gaussian_3level(64, 1)
    rk3 = W.standing_wave_2level(16)
    rk3.rk_order = 3
    rk2 = W.gaussian_3level(64, 2)
    rk2.rk_order = 2
    fd8 = W.standing_wave_2level(32)
    fd8.fd_order = 8
    uni = W.gaussian_3level(64, 0, subcycle=False)
    return [("standing wave 2-level 32^3", c1, 8, None), ("gaussian 3-level 64^3 + noise", c2, 4, 1),
            ("RK3", rk3, 6, None), ("RK2", rk2, 3, 2), ("8th order", fd8, 4, None), ("uniform step", uni, 2, 0)]


@pytest.mark.parametrize("name,h,steps,noise", _cases(), ids=[c[0] for c in _cases()])
def test_persistent_form_equals_graph_form(sc, name, h, steps, noise):
    ref, n_graph, zu_ref = _run(sc, h, sc.SC_EXEC_GRAPH, steps, noise)
    got, n_persist, zu = _run(sc, h, sc.SC_EXEC_PERSISTENT, steps, noise)
    assert n_persist == 1 and n_graph > 10
    assert zu == zu_ref
    for lg, lr in zip(got, ref):
        for g, r in zip(lg, lr):
            assert np.array_equal(g, r), name


def test_persistent_form_matches_oracle(sc, orc):
    """The configs[0] standing wave through the persistent form, 32 coarse
    steps, against the CPU oracle at the wave tolerance (1e-12)."""
    h = W.standing_wave_2level(32)
    arrays = init_arrays(h)
    ctx = sc.Context(h, exec_mode=sc.SC_EXEC_PERSISTENT)
    o = make_oracle(orc, h)
    load(ctx, h, arrays)
    load(o, h, arrays)
    ctx.sc_advance(32)
    o.advance(32)
    assert max_rel_diff(fetch(ctx, h), fetch(o, h)) <= 1e-12
    ctx.close()


def test_persistent_form_is_wave_only(sc):
    with pytest.raises(sc.SubcycError) as e:
        sc.Context(W.bl_3level(20), exec_mode=sc.SC_EXEC_PERSISTENT)
    assert e.value.code == sc.SC_EINVAL
