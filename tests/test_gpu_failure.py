"""Failure detection and recovery paths, exercised from the host side only
(no device fault is provoked): allocation failures injected through the
allocator callback and the server's pool, bounded waits that run out, and the
per-coarse-step finiteness check fed with a NaN through the public field API."""
import ctypes

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


class FailingAllocator:
    """sc_allocator over torch's caching allocator that returns NULL on its
    k-th call and counts the allocations still live."""

    def __init__(self, sc, k):
        import torch
        self.k, self.calls, self.live = k, 0, {}
        dev = torch.cuda.current_device()

        def _alloc(nbytes, user):
            self.calls += 1
            if self.calls == self.k:
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes), dev)
            self.live[p] = nbytes
            return p

        def _free(ptr, user):
            self.live.pop(ptr)
            torch.cuda.caching_allocator_delete(ptr)

        self.c = sc.sc_allocator(sc.ALLOC_FN(_alloc), sc.FREE_FN(_free), None)


@pytest.mark.parametrize("system", ["wave", "z4c"])
def test_allocation_failure_at_any_point_rolls_back(sc, system):
    """sc_create with an allocator that fails on its k-th call: SC_ENOMEM,
    and every allocation made before the failure is released, for a failure
    at the first, an intermediate and the last allocation."""
    h = W.gaussian_3level(64, 1) if system == "wave" else W.bl_3level(20)
    probe = FailingAllocator(sc, 0)
    with sc.Context(h, allocator=probe.c) as ctx:
        n_alloc = probe.calls
        fp = ctx.sc_footprint()
        assert fp > 0 and len(probe.live) > 0
    assert not probe.live and n_alloc > 3
    for k in sorted({1, 2, n_alloc // 2, n_alloc - 1, n_alloc}):
        a = FailingAllocator(sc, k)
        with pytest.raises(sc.SubcycError) as e:
            sc.Context(h, allocator=a.c)
        assert e.value.code == sc.SC_ENOMEM, (k, e.value)
        assert not a.live, (k, len(a.live))


def test_server_admission_failure(sc):
    """A request whose state cannot be allocated while nothing else runs
    fails with SC_ENOMEM and holds no memory; with another request running
    it is retried and completes once the injected failure has passed."""
    h = W.standing_wave_2level(16)
    srv = sc.Server(hbm_budget_bytes=8 << 30, max_active=4)
    srv.sc_server_inject_alloc_failure(3)
    t = srv.sc_server_submit(h, 4)
    srv.sc_server_tick()
    with pytest.raises(sc.SubcycError) as e:
        srv.sc_server_poll(t)
    assert e.value.code == sc.SC_ENOMEM
    assert srv.sc_server_stats()["bytes_in_use"] == 0
    srv.sc_server_release(t)
    long_run = srv.sc_server_submit(W.gaussian_3level(64, 0), 40)
    srv.sc_server_tick()
    srv.sc_server_inject_alloc_failure(2)
    t2 = srv.sc_server_submit(h, 4)
    srv.sc_server_tick()  # admission of t2 fails and is queued again
    assert srv.sc_server_wait(t2, 120.0) > 0
    assert srv.sc_server_wait(long_run, 120.0) > 0
    ref = sc.Context(h)
    ref.sc_set_initial_data(h.id_kind, h.id_params)
    ref.sc_advance(4)
    assert np.array_equal(srv.sc_server_read(t2, 1, 0, 0), ref.sc_get_field(1, 0, 0))
    ref.close()
    for q in (t2, long_run):
        srv.sc_server_release(q)
    assert srv.sc_server_stats()["bytes_in_use"] == 0
    srv.close()


def test_bounded_waits_run_out_and_recover(sc):
    """sc_synchronize_timeout and sc_server_wait return SC_ETIMEOUT while work
    is still queued and leave the context and the request usable."""
    h = W.gaussian_3level(128, 0)
    ctx = sc.Context(h)
    ctx.sc_set_initial_data(h.id_kind, h.id_params)
    ctx.sc_advance(20)
    with pytest.raises(sc.SubcycError) as e:
        ctx.sc_synchronize_timeout(1e-5)
    assert e.value.code == sc.SC_ETIMEOUT
    ctx.sc_synchronize_timeout(300.0)
    ctx.close()
    srv = sc.Server(hbm_budget_bytes=8 << 30, max_active=2)
    t = srv.sc_server_submit(h, 20)
    with pytest.raises(sc.SubcycError) as e:
        srv.sc_server_wait(t, 1e-5)
    assert e.value.code == sc.SC_ETIMEOUT
    assert srv.sc_server_wait(t, 300.0) > 0
    srv.sc_server_release(t)
    srv.close()


@pytest.mark.parametrize("system", ["wave", "z4c"])
def test_finite_check_after_every_coarse_step(sc, system):
    """A context created with the per-step finiteness check reports a NaN
    planted in a refined level at the next sc_synchronize (SC_ENONFINITE),
    clears the report, and a finite state passes."""
    h = W.standing_wave_2level(16) if system == "wave" else W.bl_3level(20)
    ctx = sc.Context(h, finite_check=True)
    ctx.sc_set_initial_data(h.id_kind, h.id_params)
    ctx.sc_advance(2)
    ctx.sc_synchronize()
    a = ctx.sc_get_field(1, 0, 0)
    a[2, 3, 4] = np.nan
    ctx.sc_set_field(1, 0, 0, a)
    ctx.sc_advance(1)
    with pytest.raises(sc.SubcycError) as e:
        ctx.sc_synchronize()
    assert e.value.code == sc.SC_ENONFINITE
    ctx.sc_synchronize()  # reported once, then cleared
    ctx.sc_set_initial_data(h.id_kind, h.id_params)
    ctx.sc_advance(1)
    ctx.sc_synchronize()
    ctx.close()
