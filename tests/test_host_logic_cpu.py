"""Host logic of the C ABI that needs no GPU: descriptor validation and the
device-footprint estimate used for admission by the server (no CUDA call is
made)."""
import pytest

from paper_2503_09629_gb300 import workloads as W


@pytest.fixture(scope="module")
def sc():
    import paper_2503_09629_gb300 as m
    from paper_2503_09629_gb300 import buildlib
    buildlib.build()
    return m


def test_footprint_estimate_follows_the_options(sc):
    h = W.bl_7level()
    base = sc.sc_footprint_estimate(h)
    # 7 levels, 22 fields, 8 arrays per level over about 2.5e6 cells plus ghosts and scratch: several GB
    assert 4e9 < base < 12e9
    h.fd_order = 8  # 4 ghost layers instead of 3
    assert sc.sc_footprint_estimate(h) > base
    h.fd_order, h.rk_order = 4, 2  # two stage vectors instead of four
    assert sc.sc_footprint_estimate(h) < base
    h.rk_order = 3  # three, plus k4 on the levels that have a finer level
    rk3 = sc.sc_footprint_estimate(h)
    assert sc.sc_footprint_estimate(W.Hierarchy(**{**h.__dict__, "rk_order": 2})) < rk3 < base
    small = W.bl_3level(20)
    assert sc.sc_footprint_estimate(small) < base / 20


@pytest.mark.parametrize("field,value,msg", [("fd_order", 6, "fd_order"), ("rk_order", 5, "rk_order"),
                                             ("rk_order", 1, "rk_order"), ("cfl", 0.0, "cfl")])
def test_invalid_descriptors_are_rejected_with_a_message(sc, field, value, msg):
    h = W.standing_wave_2level(16)
    setattr(h, field, value)
    with pytest.raises(sc.SubcycError) as e:
        sc.sc_footprint_estimate(h)
    assert e.value.code == -1 and msg in str(e.value)


def test_no_cpu_fallback_when_the_library_cannot_be_built(tmp_path):
    """The product path has no CPU fallback: with no library and no nvcc the
    binding raises instead of computing anything (run in a subprocess with
    the library path pointed at an empty directory and nvcc hidden)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = (
        "import sys, shutil\n"
        f"sys.path.insert(0, {root!r})\n"
        "import paper_2503_09629_gb300 as m\n"
        "from paper_2503_09629_gb300 import buildlib\n"
        f"m.LIB_PATH = {str(tmp_path / 'missing.so')!r}\n"
        "shutil.which = lambda name, *a, **k: None\n"
        "buildlib.nvcc = lambda: (_ for _ in ()).throw(RuntimeError('nvcc not found'))\n"
        "try:\n"
        "    m.lib()\n"
        "except Exception as e:\n"
        "    print('raised', type(e).__name__)\n"
        "    sys.exit(0)\n"
        "sys.exit(3)\n")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "raised" in r.stdout, (r.stdout, r.stderr)
