"""Pins of the oracle's RK2 and RK3 subcycling (the extension that Sec. V of
the paper leaves to future work).  The methods are the explicit midpoint
rule (RK2) and Heun's third-order method (RK3); the tests take them from
their Butcher tableaux (RK3's dense output also reads k4 = f(y_{n+1})) and
check the oracle's dense output and stage reconstruction against exact
solutions, measured orders and exactness on nilpotent systems -- never
against the oracle's own formulas.
"""
import numpy as np
import pytest
import scipy.linalg

from paper_2503_09629_gb300 import workloads as W

# Butcher tableaux (A strictly lower triangular, b, c).
TABLEAU = {
    2: (np.array([[0.0, 0.0], [0.5, 0.0]]), np.array([0.0, 1.0])),
    3: (np.array([[0.0, 0.0, 0.0], [1 / 3, 0.0, 0.0], [0.0, 2 / 3, 0.0]]), np.array([0.25, 0.0, 0.75])),
}


def make(orc, h, **over):
    kw = h.kwargs()
    kw.update(over)
    return orc.Oracle(h.system, h.boxes, h.ncells0, h.origin, h.h0, **kw)


def rk_stages(rk, L, y, H):
    """Stage states Y_i and stage vectors k_i of one step of y' = L y."""
    A, _ = TABLEAU[rk]
    Ys, ks = [], []
    for i in range(len(A)):
        Yi = y + H * sum(A[i, j] * ks[j] for j in range(i))
        Ys.append(Yi)
        ks.append(L @ Yi)
    return Ys, np.stack(ks)


def dense_inputs(rk, L, y, H):
    """The stage vectors the dense output reads: k1, k2 (RK2); k1, k2, k3 and
    k4 = f(y_{n+1}) (RK3)."""
    _, K = rk_stages(rk, L, y, H)
    if rk == 3:
        _, b = TABLEAU[rk]
        K = np.vstack([K, L @ (y + H * (b @ K))])
    return K


# local order of the dense output (error ~ H^p) and of the stage reconstruction
DENSE_ORDER = {2: 3, 3: 4}


def recon(orc, rk, yn, K, H, th0, which):
    return np.array([orc.amr_value(yn[c], K[:, c], H, th0, which, rk=rk) for c in range(len(yn))])


@pytest.mark.parametrize("rk", [2, 3])
def test_dense_output_reproduces_the_step(orc, rk):
    """theta = 1 gives the method's weights b, theta = 0 gives 0,
    sum_i b_i(theta) = theta, and the first derivative at theta = 0 is k1."""
    _, b = TABLEAU[rk]
    np.testing.assert_allclose(orc.dense_b(1.0, 0, rk)[:rk], b, atol=1e-15)
    np.testing.assert_allclose(orc.dense_b(0.0, 0, rk), 0.0, atol=0)
    for th in np.linspace(0, 1, 11):
        assert abs(orc.dense_b(th, 0, rk).sum() - th) < 1e-15
    np.testing.assert_allclose(orc.dense_b(0.0, 1, rk)[:rk], np.eye(rk)[0], atol=0)


@pytest.mark.parametrize("rk,m", [(2, 1), (2, 2), (3, 1), (3, 2), (3, 3)])
def test_dense_output_derivative_weights(orc, rk, m):
    """m-th theta-derivative weights against a centred difference of the
    (m-1)-th; the weights are polynomials of degree rk (quadratic, cubic)."""
    eps = 1e-5
    for th in (0.1, 0.37, 0.5, 0.8):
        num = (orc.dense_b(th + eps, m - 1, rk) - orc.dense_b(th - eps, m - 1, rk)) / (2 * eps)
        np.testing.assert_allclose(orc.dense_b(th, m, rk), num, atol=1e-8)
    np.testing.assert_allclose(orc.dense_b(0.3, rk + 1, rk), 0, atol=0)


@pytest.mark.parametrize("rk", [2, 3])
def test_dense_output_order(orc, rk):
    """Dense output y_n + H sum_i b_i(theta) k_i against the exact flow of a
    damped oscillator: the error at interior theta falls as H^3 for RK2
    (second-order extension) and H^4 for RK3 (cubic Hermite)."""
    L = np.array([[-0.3, 1.0], [-1.0, -0.1]])
    yn = np.array([0.7, -0.4])
    errs = []
    for H in (0.2, 0.1, 0.05):
        K = dense_inputs(rk, L, yn, H)
        e = 0.0
        for th in (0.37, 0.5, 0.81):
            b = orc.dense_b(th, 0, rk)[:len(K)]
            y = yn + H * (b @ K)
            e = max(e, np.abs(y - scipy.linalg.expm(th * H * L) @ yn).max())
        errs.append(e)
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > DENSE_ORDER[rk] - 0.2), orders


@pytest.mark.parametrize("rk", [2, 3])
@pytest.mark.parametrize("theta0", [0.0, 0.5])
def test_stage_reconstruction_exact_for_nilpotent_system(orc, rk, theta0):
    """For y' = L y with L^rk+1 = 0 the solution is a polynomial of degree rk
    in t that the method integrates exactly and the dense output (quadratic
    for RK2, cubic Hermite for RK3) reproduces: the reconstructed fine stage
    states must equal the true fine stages (step h = H/2 from the exact state
    at theta0) and the end-of-substep value the exact state."""
    rng = np.random.default_rng(11)
    L = np.diag(rng.uniform(0.5, 2.0, rk), 1)  # (rk+1)^2, L^(rk+1) = 0
    yn = rng.normal(size=rk + 1)
    H = 0.41
    K = dense_inputs(rk, L, yn, H)
    y0 = scipy.linalg.expm(theta0 * H * L) @ yn
    true, _ = rk_stages(rk, L, y0, H / 2)
    for i in range(rk):
        np.testing.assert_allclose(recon(orc, rk, yn, K, H, theta0, i + 1), true[i], rtol=1e-13, atol=1e-13)
    end = scipy.linalg.expm((theta0 + 0.5) * H * L) @ yn
    np.testing.assert_allclose(recon(orc, rk, yn, K, H, theta0, 0), end, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("rk", [2, 3])
def test_stage_reconstruction_order_for_general_system(orc, rk):
    """General linear system: the stage reconstruction error falls with the
    dense output's local order (H^3 for RK2, H^4 for RK3)."""
    rng = np.random.default_rng(12)
    L = rng.normal(size=(5, 5))
    yn = rng.normal(size=5)
    errs = []
    for H in (0.1, 0.05, 0.025):
        e = 0.0
        for th0 in (0.0, 0.5):
            K = dense_inputs(rk, L, yn, H)
            true, _ = rk_stages(rk, L, scipy.linalg.expm(th0 * H * L) @ yn, H / 2)
            for i in range(rk):
                e = max(e, np.abs(recon(orc, rk, yn, K, H, th0, i + 1) - true[i]).max())
        errs.append(e)
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > DENSE_ORDER[rk] - 0.2), orders


def _poly(X, Y, Z, coef):
    out = np.zeros_like(X)
    for (a, b, c), v in coef.items():
        out += v * X ** a * Y ** b * Z ** c
    return out


def _lap(coef):
    out = {}
    for (a, b, c), v in coef.items():
        for d, e in enumerate((a, b, c)):
            if e >= 2:
                m = [a, b, c]
                m[d] -= 2
                out[tuple(m)] = out.get(tuple(m), 0.0) + v * e * (e - 1)
    return out


@pytest.mark.parametrize("rk", [2, 3])
def test_subcycling_exact_for_polynomial_wave(orc, rk):
    """Whole subcycled scheme with RK2 / RK3 on data where every
    approximation is exact: u of total degree rk and Pi of degree rk - 1 make
    the wave system nilpotent (L^(rk+1) = 0), the method integrates it
    exactly, its dense output reproduces it, and quintic transfer and the
    4th-order Laplacian are exact on such polynomials.  Three levels, three
    coarse steps."""
    rng = np.random.default_rng(21)
    mons = lambda deg: [(a, b, c) for a in range(4) for b in range(4) for c in range(4) if a + b + c <= deg]
    cu = {m: rng.normal() for m in mons(rk)}
    cp = {m: rng.normal() for m in mons(rk - 1)}
    # jets y, L y, L^2 y, L^3 y of L(u, Pi) = (Pi, Lap u), as coefficient dicts
    jet_c = [(cu, cp)]
    for _ in range(3):
        u, p = jet_c[-1]
        jet_c.append((p, _lap(u)))

    def jets(X, Y, Z):
        return [np.stack([_poly(X, Y, Z, u), _poly(X, Y, Z, p)]) for u, p in jet_c]

    def exact(t, X, Y, Z):
        J = jets(X, Y, Z)
        return J[0] + t * J[1] + t ** 2 / 2 * J[2] + t ** 3 / 6 * J[3]

    A, _ = TABLEAU[rk]

    def bc(which, t_n, dt, xyz):
        X, Y, Z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
        if which == 0:
            return exact(t_n + dt, X, Y, Z)
        J = jets(X, Y, Z)
        # jets at t_n (L^4 = 0 for both data sets)
        Jn = [J[0] + t_n * J[1] + t_n ** 2 / 2 * J[2] + t_n ** 3 / 6 * J[3],
              J[1] + t_n * J[2] + t_n ** 2 / 2 * J[3], J[2] + t_n * J[3], J[3]]
        # stage states as combinations sum_m a_m L^m y_n (L shifts the jet)
        coef = []
        for i in range(which):
            a = np.array([1.0, 0.0, 0.0, 0.0])
            for j in range(i):
                kj = np.concatenate([[0.0], coef[j][:3]])
                a = a + dt * A[i, j] * kj
            coef.append(a)
        a = coef[which - 1]
        return sum(a[m] * Jn[m] for m in range(4))

    boxes = [[W.cube(0, 24)], [W.cube(12, 24)], [W.cube(36, 24)]]
    h = W.Hierarchy(system=W.WAVE, boxes=boxes, ncells0=(24, 24, 24), origin=(-0.75, -0.75, -0.75),
                    h0=1.0 / 16, bc=2, rk_order=rk)
    o = make(orc, h)
    o.set_bc_callback(bc)
    for l in range(3):
        X, Y, Z = h.cell_centres(l, 0, ghosted=True)
        y = exact(0.0, X, Y, Z)
        o.set_field(l, 0, 0, y[0], ghosted=True)
        o.set_field(l, 0, 1, y[1], ghosted=True)
    o.advance(3)
    t = o.time
    for l in range(3):
        X, Y, Z = h.cell_centres(l, 0)
        ex = exact(t, X, Y, Z)
        for f in range(2):
            err = np.abs(o.get_field(l, 0, f) - ex[f]).max() / np.abs(ex[f]).max()
            assert err < 1e-12, (rk, l, f, err)


def _standing_error(orc, n, rk, subcycle=True, t_end=0.25):
    h = W.standing_wave_2level(n, subcycle=subcycle)
    h.rk_order = rk
    o = make(orc, h)
    o.set_initial_data(h.id_kind, h.id_params)
    o.advance(int(round(t_end / (h.cfl * h.h0))))
    om = 2 * np.sqrt(3) * np.pi
    err = 0.0
    for l in range(2):
        X, Y, Z = h.cell_centres(l, 0)
        s = np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y) * np.sin(2 * np.pi * Z)
        err = max(err, np.abs(o.get_field(l, 0, 0) - s * np.cos(om * o.time)).max())
    return err, o


@pytest.mark.parametrize("rk,lo,hi", [(3, 2.7, 3.4), (2, 1.8, 2.3)])
def test_standing_wave_converges_at_the_method_order(orc, rk, lo, hi):
    """Sec. IV.A test with the lower-order methods: the subcycled error
    against the exact standing wave converges at the order of the time
    integrator (the 4th-order space error is smaller here)."""
    errs = [_standing_error(orc, n, rk)[0] for n in (16, 32)]
    order = np.log2(errs[0] / errs[1])
    assert lo < order < hi, (errs, order)
