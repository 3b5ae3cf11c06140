"""The seeded workloads have the geometry the benchmark and parity cases are
named for (no method arithmetic is involved)."""
from paper_2503_09629_gb300 import workloads as W


def test_benchmark_hierarchy_geometry():
    """7-level Z4c Brill-Lindquist benchmark: [-32,32]^3 at h = 1 with 64^3
    cells, finest h = 1/64, 2,490,368 interior cells; per coarse step
    60,555,264 actual and 159,383,552 finest-equivalent cell updates."""
    h = W.bl_7level()
    assert h.nlevels == 7 and h.system == W.Z4C and h.bc == W.BC_RADIATIVE
    assert tuple(h.ncells0) == (64, 64, 64) and h.h0 == 1.0 and tuple(h.origin) == (-32.0, -32.0, -32.0)
    assert sum(h.interior_cells(l) for l in range(7)) == 2_490_368
    fin, act = h.zone_updates_per_coarse_step()
    assert (fin, act) == (159_383_552, 60_555_264)
    assert len(h.boxes[6]) == 2  # one finest box per puncture
    assert h.id_params[:4] == [0.5, 0.0, 0.0, 1.0] and h.id_params[4:] == [0.5, 0.0, 0.0, -1.0]


def test_standing_wave_and_gaussian_cases():
    h = W.standing_wave_2level(32)
    assert h.nlevels == 2 and sum(h.interior_cells(l) for l in range(2)) == 2 * 32 ** 3
    assert h.boxes[1] == [((16, 16, 16), (47, 47, 47))]  # fine box over [0.25, 0.75]^3
    g = W.gaussian_3level(64, 0)
    assert len(g.boxes[0]) == 27 and all(6 <= len(g.boxes[l]) <= 20 for l in (1, 2))
    # seeded: the same seed gives the same boxes, another seed different ones
    assert W.gaussian_3level(64, 0).boxes == g.boxes and W.gaussian_3level(64, 1).boxes != g.boxes


def test_serving_ensemble_mix():
    reqs = W.serving_requests(256, seed=0, burst=True)
    n_wave = sum(1 for _, h, _ in reqs if h.system == W.WAVE)
    assert len(reqs) == 256 and 0.5 < n_wave / 256 < 0.7
    assert all(t == 0.0 for t, _, _ in reqs)
    pois = W.serving_requests(64, seed=0, burst=False, mean_interarrival=0.1)
    times = [t for t, _, _ in pois]
    assert times == sorted(times) and times[-1] > 0
