"""Pins of the oracle's macro charge-density schedules (Sec. VI): each model,
its schedule and its bin integrals against closed forms, limits and
independent quadrature (scipy, numpy)."""
import math

import numpy as np
import pytest

import oracle

scipy_integrate = pytest.importorskip("scipy.integrate")


@pytest.mark.parametrize("n", [1, 2, 5, 8, 16, 24])
def test_gauss_legendre_against_numpy(n):
    x, w = oracle.gauss_legendre(n)
    nx, nw = np.polynomial.legendre.leggauss(n)
    assert np.allclose(np.sort(x), np.sort(nx), atol=1e-14)
    assert np.allclose(w[np.argsort(x)], nw[np.argsort(nx)], atol=1e-14)
    # exact for polynomials of degree 2n - 1
    for d in range(2 * n):
        assert np.sum(w * x ** d) == pytest.approx(0.0 if d % 2 else 2.0 / (d + 1), abs=1e-13)


def test_eta_schedule_endpoints_and_blend():
    rp = oracle.rho_params()
    T = rp.T
    eta_b0 = math.sqrt(2 * math.log(2)) / rp.beta_min       # scheme B at alpha = 0
    eta_a1 = math.sqrt(-2 * math.log(rp.r1))                 # scheme A at alpha = 1
    assert oracle.rho_eta(rp, 0) == pytest.approx(eta_b0, rel=1e-15)
    assert oracle.rho_eta(rp, T) == pytest.approx(eta_a1, rel=1e-15)
    # pure scheme B below alpha0, pure scheme A above alpha1
    t = int(0.2 * T)
    beta = rp.beta_min + (rp.beta_max - rp.beta_min) * t / T
    assert oracle.rho_eta(rp, t) == pytest.approx(math.sqrt(2 * math.log(2)) / beta, rel=1e-14)
    t = int(0.8 * T)
    a = t / T
    ea = math.sqrt(-2 * ((1 - a) * math.log(rp.r0) + a * math.log(rp.r1)))
    assert oracle.rho_eta(rp, t) == pytest.approx(ea, rel=1e-14)
    # the midpoint of the blend: smoothstep weight 1/2 -> geometric mean
    t = T // 2
    a = t / T
    ea = math.sqrt(-2 * ((1 - a) * math.log(rp.r0) + a * math.log(rp.r1)))
    eb = math.sqrt(2 * math.log(2)) / (rp.beta_min + (rp.beta_max - rp.beta_min) * a)
    assert oracle.rho_eta(rp, t) == pytest.approx(math.sqrt(ea * eb), rel=1e-14)


def test_sigma_and_k_schedules():
    rp = oracle.rho_params()
    T = rp.T
    assert oracle.rho_sigma(rp, 0) == 0.0 and math.isinf(oracle.rho_sigma(rp, T))
    s = [oracle.rho_sigma(rp, t) for t in range(0, T)]
    assert all(b > a for a, b in zip(s, s[1:]))
    assert oracle.rho_sigma(rp, 100) == pytest.approx(-rp.sigma_factor * T * math.log(1 - 100 / T))
    assert math.isinf(oracle.rho_k(rp, 0)) and oracle.rho_k(rp, T) == 0.0
    assert oracle.rho_k(rp, T // 2) == pytest.approx(rp.k_factor / math.tan(math.pi / 4))


@pytest.mark.parametrize("t", [0, 30, 150, 270, 300])
def test_gaussian_integrates_to_the_macro_area(t):
    rp = oracle.rho_params(model=oracle.RHO_GAUSS)
    w, h = 37.0, 12.5
    assert oracle.rho_integral(rp, t, w, h, -w, w, -h, h) == pytest.approx(w * h, rel=1e-13)
    # and its value at the centre is the normalization
    eta = oracle.rho_eta(rp, t)
    norm = 2 * eta ** 2 / (math.pi * math.erf(eta / math.sqrt(2)) ** 2)
    assert oracle.rho_value(rp, t, 0.0, 0.0, w, h) == pytest.approx(norm, rel=1e-14)
    assert oracle.rho_value(rp, t, 0.51 * w, 0.0, w, h) == 0.0


@pytest.mark.parametrize("model,t,tol", [
    (oracle.RHO_GAUSS, 60, 1e-10), (oracle.RHO_EXP, 150, 1e-7), (oracle.RHO_EXP, 280, 1e-7),
    (oracle.RHO_SIGMOID, 100, 1e-6), (oracle.RHO_SIGMOID, 250, 1e-6),
    (oracle.RHO_LINEAR, 200, 2e-3), (oracle.RHO_LINEAR, 290, 1e-6)])
def test_sub_rectangle_integrals_against_adaptive_quadrature(model, t, tol):
    rp = oracle.rho_params(model=model, panels=8, nodes=12)
    w, h = 20.0, 14.0
    ax, bx, ay, by = -3.0, 9.5, -7.0, 2.0  # a bin partly outside the macro
    got = oracle.rho_integral(rp, t, w, h, ax, bx, ay, by)
    ref, _ = scipy_integrate.dblquad(lambda y, x: oracle.rho_value(rp, t, x, y, w, h),
                                     max(ax, -w / 2), min(bx, w / 2), max(ay, -h / 2),
                                     min(by, h / 2), epsabs=1e-12, epsrel=1e-11)
    assert got == pytest.approx(ref, rel=tol, abs=tol * w * h)


@pytest.mark.parametrize("model", [oracle.RHO_EXP, oracle.RHO_LINEAR, oracle.RHO_SIGMOID])
def test_restoration_limits(model):
    rp = oracle.rho_params(model=model)
    w, h = 10.0, 6.0
    # fully restored at t = T: the macro's area; nothing at t = 0
    assert oracle.rho_integral(rp, rp.T, w, h, -w, w, -h, h) == pytest.approx(w * h, rel=1e-13)
    assert oracle.rho_integral(rp, 0, w, h, -w, w, -h, h) == 0.0
    # restoration grows with t
    vals = [oracle.rho_integral(rp, t, w, h, -w, w, -h, h) for t in (30, 100, 200, 290)]
    assert all(b > a for a, b in zip(vals, vals[1:]))


def test_bins_partition_the_macros():
    rp = oracle.rho_params(model=oracle.RHO_GAUSS)
    mx, my = np.array([30.0, 71.3]), np.array([40.0, 22.2])
    mw, mh = np.array([17.0, 9.0]), np.array([11.0, 23.0])
    rho = oracle.macro_density(rp, 120, mx, my, mw, mh, (0.0, 0.0, 100.0, 80.0), 10, 8)
    assert rho.sum() == pytest.approx(float((mw * mh).sum()), rel=1e-12)
    assert (rho >= 0).all()
    # a bin far from both macros gets nothing
    assert rho[0] == 0.0
    # mirror symmetry of one macro centred in a bin
    r2 = oracle.macro_density(rp, 120, [55.0], [45.0], [20.0], [10.0], (0.0, 0.0, 100.0, 80.0), 10, 8)
    g = r2.reshape(8, 10)
    assert np.allclose(g[:, 4], g[:, 6], rtol=1e-12) and np.allclose(g[3], g[5], rtol=1e-12)
