"""Served form (continuous batching of independent evolutions): every
request's result is bitwise the same alone and in a mix where requests queue
for slots and memory and run concurrently; admission respects the memory
budget; the plain per-box execution form gives bitwise the same fields as the
graph form."""
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


def _mix():
    reqs = W.serving_requests(10, seed=3, burst=True)
    # keep the test short: small Z4c boxes, few steps
    out = []
    for i, (_t, h, steps) in enumerate(reqs):
        if h.system == W.Z4C:
            h = W.bl_3level(20 + 4 * (i % 2), 0.4 + 0.02 * i, 0.5, 2.0 + 0.1 * i)
            steps = 2
        else:
            steps = min(steps, 12)
        out.append((h, steps))
    return out


def _fields(getf, h):
    return [np.stack([getf(l, b, f) for f in range(h.nfields())]) for l in range(h.nlevels)
            for b in range(len(h.boxes[l]))]


def test_alone_equals_in_mix(sc):
    mix = _mix()
    alone = []
    for h, steps in mix:
        srv = sc.Server(hbm_budget_bytes=64 << 30, max_active=1)
        t = srv.sc_server_submit(h, steps)
        srv.run_until_done([t], timeout_s=120.0)
        alone.append(_fields(lambda l, b, f: srv.sc_server_read(t, l, b, f), h))
        srv.close()
    # a budget that holds only a few requests at once, and fewer slots than requests
    budget = sorted(sc.sc_footprint_estimate(h) for h, _ in mix)[-3:]
    srv = sc.Server(hbm_budget_bytes=sum(budget), max_active=4)
    tickets = [srv.sc_server_submit(h, s) for h, s in mix]
    index = {t: i for i, t in enumerate(tickets)}
    got = {}

    def on_done(t):  # a client reads a finished request and releases it
        h = mix[index[t]][0]
        got[t] = _fields(lambda l, b, f: srv.sc_server_read(t, l, b, f), h)
        done, lat = srv.sc_server_poll(t)
        assert done and lat > 0
        srv.sc_server_release(t)

    active, queued, _ = srv.sc_server_tick()
    assert active >= 2 and queued >= 1  # concurrent requests, and some waiting for slots or memory
    srv.run_until_done(tickets, timeout_s=300.0, on_done=on_done)
    for t, ref in zip(tickets, alone):
        for a, b in zip(got[t], ref):
            assert np.array_equal(a, b)
    assert srv.sc_server_stats()["bytes_in_use"] == 0
    srv.close()


def test_request_larger_than_budget_refused(sc):
    srv = sc.Server(hbm_budget_bytes=1 << 20, max_active=2)
    with pytest.raises(sc.SubcycError) as e:
        srv.sc_server_submit(W.bl_3level(24), 1)
    assert e.value.code == sc.SC_EBUSY
    srv.close()


@pytest.mark.parametrize("system", ["wave", "z4c"])
def test_per_box_form_equals_graph_form(sc, system):
    h = W.gaussian_3level(64, 2) if system == "wave" else W.bl_3level(24)
    res = []
    for mode in (sc.SC_EXEC_GRAPH, sc.SC_EXEC_PER_BOX):
        c = sc.Context(h, exec_mode=mode)
        c.sc_set_initial_data(h.id_kind, h.id_params)
        c.sc_advance(2)
        res.append(_fields(lambda l, b, f: c.sc_get_field(l, b, f), h))
        c.close()
    for a, b in zip(*res):
        assert np.array_equal(a, b)


def test_merged_launches_equal_per_request_graphs(sc):
    """Merged form (scalar-wave requests of a tick in one persistent launch)
    against one graph per request on its own stream: bitwise the same
    fields for every request of the mix; the merged server launches fewer
    kernels."""
    mix = _mix()
    res, launches = {}, {}
    for merge in (False, True):
        srv = sc.Server(hbm_budget_bytes=64 << 30, max_active=8)
        srv.sc_server_set_merge(merge)
        tickets = [srv.sc_server_submit(h, s) for h, s in mix]
        got = {}

        def on_done(t, srv=srv, got=got, tickets=tickets):
            h = mix[tickets.index(t)][0]
            got[t] = _fields(lambda l, b, f: srv.sc_server_read(t, l, b, f), h)
            srv.sc_server_release(t)

        srv.run_until_done(tickets, timeout_s=300.0, on_done=on_done)
        res[merge] = [got[t] for t in tickets]
        launches[merge] = srv.sc_server_stats()["launches"]
        srv.close()
    for a, b in zip(res[False], res[True]):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    assert launches[True] < launches[False]
