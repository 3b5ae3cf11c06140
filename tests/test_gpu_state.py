"""Whole-state transfer (sc_set_state / sc_get_state): the packed layout
matches the per-field calls bitwise, in both directions, from numpy and from
page-locked buffers."""
import numpy as np
import pytest

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


def _per_field(ctx, h, ghosted_level0):
    parts = []
    for l in range(h.nlevels):
        for b in range(len(h.boxes[l])):
            for f in range(h.nfields()):
                parts.append(ctx.sc_get_field(l, b, f, ghosted=bool(ghosted_level0 and l == 0)).ravel())
    return np.concatenate(parts)


@pytest.mark.parametrize("ghosted_level0", [False, True])
def test_state_matches_per_field_calls(sc, ghosted_level0):
    h = W.bl_3level(20)
    ctx = sc.Context(h)
    ctx.sc_set_initial_data(h.id_kind, h.id_params)
    ctx.sc_advance(1)
    ref = _per_field(ctx, h, ghosted_level0)
    assert ctx.sc_state_bytes(ghosted_level0) == ref.nbytes
    got = ctx.sc_get_state(ghosted_level0=ghosted_level0)
    assert np.array_equal(got, ref)
    # write a perturbed state back and read it through the per-field calls
    new = ref * (1.0 + 1e-3 * np.sin(np.arange(ref.size)))
    ctx.sc_set_state(new, ghosted_level0=ghosted_level0)
    assert np.array_equal(_per_field(ctx, h, ghosted_level0), new)
    ctx.close()


def test_state_through_pinned_buffers_and_uneven_boxes(sc):
    torch = pytest.importorskip("torch")
    h = W.gaussian_3level(64, 1)
    ctx = sc.Context(h)
    ctx.sc_set_initial_data(h.id_kind, h.id_params)
    n = ctx.sc_state_bytes() // 8
    buf = torch.empty(n, dtype=torch.float64).pin_memory()
    ctx.sc_get_state(buf.data_ptr())
    ref = _per_field(ctx, h, False)
    assert np.array_equal(buf.numpy(), ref)
    buf.mul_(2.0)
    ctx.sc_set_state(buf.data_ptr())
    assert np.array_equal(_per_field(ctx, h, False), 2.0 * ref)
    ctx.close()


def test_direct_and_staged_transfers_agree(sc):
    """Both transfer forms move the same bytes: the direct form (kernels read
    and write page-locked host memory through its device mapping, no DMA) and
    the staged form (one DMA to a device staging buffer plus kernels); the
    event-timed split of each is reported, and the direct form refuses
    pageable memory."""
    torch = pytest.importorskip("torch")
    h = W.bl_3level(20)
    ctx = sc.Context(h)
    ctx.sc_set_initial_data(h.id_kind, h.id_params)
    ctx.sc_advance(1)
    ref = ctx.sc_get_state(ghosted_level0=True)  # numpy (pageable): staged
    st = ctx.sc_transfer_stats()
    assert not st["direct"] and st["bytes"] == ref.nbytes and st["copy_ms"] > 0
    pinned_ref = torch.from_numpy(ref).pin_memory()
    buf = torch.empty(ref.size, dtype=torch.float64).pin_memory()
    for mode, direct in ((sc.SC_XFER_AUTO, True), (sc.SC_XFER_STAGED, False), (sc.SC_XFER_DIRECT, True)):
        ctx.sc_set_transfer_mode(mode)
        buf.zero_()
        ctx.sc_get_state(buf.data_ptr(), ghosted_level0=True)
        st = ctx.sc_transfer_stats()
        assert st["direct"] == direct and st["bytes"] == ref.nbytes, (mode, st)
        assert (st["copy_ms"] == 0.0) == direct and st["kernel_ms"] > 0, (mode, st)
        assert np.array_equal(buf.numpy(), ref), mode
        buf.mul_(3.0)
        ctx.sc_set_state(buf.data_ptr(), ghosted_level0=True)
        assert ctx.sc_transfer_stats()["direct"] == direct
        buf.zero_()
        ctx.sc_get_state(buf.data_ptr(), ghosted_level0=True)
        assert np.array_equal(buf.numpy(), 3.0 * ref), mode
        ctx.sc_set_state(pinned_ref.data_ptr(), ghosted_level0=True)
    with pytest.raises(sc.SubcycError) as e:
        ctx.sc_get_state(np.empty_like(ref), ghosted_level0=True)  # pageable memory in the direct form
    assert e.value.code == sc.SC_EINVAL
    ctx.close()


@pytest.mark.parametrize("make", [lambda: W.bl_3level(20), lambda: W.gaussian_3level(64, 2)])
def test_checkpoint_restart_continues_bitwise(sc, make):
    """Checkpoint/restart through the public API: the whole state read after
    three coarse steps and written into a fresh context continues exactly
    like the original (each coarse step recomputes all stage vectors and
    ghost values from the state)."""
    h = make()
    g0 = h.bc == W.BC_RADIATIVE  # the evolved ghost shell of level 0 is state
    a = sc.Context(h)
    a.sc_set_initial_data(h.id_kind, h.id_params)
    a.sc_advance(3)
    snap = a.sc_get_state(ghosted_level0=g0)
    with sc.Context(h) as b:
        b.sc_set_state(snap, ghosted_level0=g0)
        a.sc_advance(2)
        b.sc_advance(2)
        assert np.array_equal(a.sc_get_state(ghosted_level0=g0), b.sc_get_state(ghosted_level0=g0))
    a.close()
