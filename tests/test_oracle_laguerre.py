"""Pins of the Laguerre-chain oracle (Section 4.1, Eqs. series_lag and
laguerre_h) against things other than itself: exact factorials, SciPy's
generalised Laguerre polynomials, the orthonormality of the Laguerre
functions, and the transform of a second time derivative computed by
quadrature from the definition of the coefficients."""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy import integrate, special

import oracle as O
from oracle import laguerre as L


@pytest.mark.parametrize("alpha", [2, 5])
def test_weights_are_the_factorial_ratios(alpha):
    for m in range(0, 40):
        a, w = L.weights(m, alpha)
        exact = Fraction(math.factorial(m), math.factorial(m + alpha))
        assert a * a == pytest.approx(float(exact), rel=1e-13)
        assert w * w == pytest.approx(float(1 / exact), rel=1e-13)


@pytest.mark.parametrize("m", [0, 1, 2, 7, 15])
def test_laguerre_function_matches_scipy_polynomials(m):
    alpha = 5
    y = np.linspace(0.0, 40.0, 81)
    ref = math.sqrt(math.factorial(m) / math.factorial(m + alpha)) * y ** (alpha / 2) * np.exp(-y / 2) * \
        special.eval_genlaguerre(m, alpha, y)
    assert np.allclose(L.laguerre_function(m, alpha, y), ref, rtol=1e-11, atol=1e-14)


def test_laguerre_functions_are_orthonormal():
    alpha, h = 5, 3.0
    for m in range(5):
        for n in range(5):
            v, _ = integrate.quad(lambda t: h * L.laguerre_function(m, alpha, h * t) *
                                  L.laguerre_function(n, alpha, h * t), 0, 80, limit=400)
            assert v == pytest.approx(1.0 if m == n else 0.0, abs=1e-10)


def test_second_derivative_coefficients_match_quadrature_of_the_definition():
    """u(t) = t^3 exp(-t) (at rest at t = 0): the coefficients of u'' by
    quadrature of Eq. series_lag equal the oracle's expression in those of u."""
    alpha, h = 5, 3.0

    def coef(fun, m):
        g = lambda t: fun(t) * (h * t) ** (-alpha / 2) * math.sqrt(h) * L.laguerre_function(m, alpha, h * t)
        return integrate.quad(g, 0, 60, limit=400, epsabs=1e-14, epsrel=1e-12)[0]

    u = lambda t: t ** 3 * np.exp(-t)
    u2 = lambda t: (6 * t - 6 * t ** 2 + t ** 3) * np.exp(-t)
    Q = [coef(u, k) for k in range(10)]
    got = L.second_derivative_coefficients(Q, h, alpha)
    want = [coef(u2, m) for m in range(10)]
    assert np.allclose(got, want, rtol=1e-9, atol=1e-13)


def test_harmonic_rhs_is_source_minus_the_time_term():
    """f_m src - c2 a_m sum (m - k) w_k Q_k equals f_m src - (c2 / h^2)
    ([u_tt]_m - h^2/4 Q_m) for arbitrary fields, and is f_0 src at m = 0."""
    rng = np.random.default_rng(0)
    alpha, h = 5, 7.0
    Q = [rng.normal(size=(3, 4)) for _ in range(6)]
    c2, src = rng.uniform(1, 2, size=(3, 4)), rng.normal(size=(3, 4))
    utt = L.second_derivative_coefficients(Q, h, alpha)
    for m in range(6):
        got = L.harmonic_rhs(m, Q[:m], c2, src, 0.3 * m + 1, alpha)
        want = (0.3 * m + 1) * src - c2 / h ** 2 * (utt[m] - h * h / 4 * Q[m])
        assert np.allclose(got, want, rtol=1e-12, atol=1e-12)
    assert np.array_equal(L.harmonic_rhs(0, [], c2, src, 2.0, alpha), 2.0 * src)


def test_chain_solves_each_harmonic_with_its_own_right_hand_side():
    nr, nz = 12, 10
    g = O.Grid(nr, nz, lr=1.0, lz=0.8, bc_z=1)
    rng = np.random.default_rng(1)
    kr, kz = rng.uniform(1, 2, size=(nr, nz)), rng.uniform(1, 2, size=(nr, nz + 1))
    c2 = np.full((nr, nz), 40.0)
    op = O.Operator(kr, kz, c2 / 4.0, g)
    src = np.zeros((nr, nz))
    src[0, 0] = 1.0
    fm = [1.0, -0.5, 0.25, 0.1]
    Q = L.chain(lambda rhs, prev: op.solve(rhs, 1e-12)[0], c2, src, fm, 5)
    for m in range(4):
        phi = op.phi(L.harmonic_rhs(m, Q[:m], c2, src, fm[m], 5))
        assert np.linalg.norm(op.apply_A(Q[m]) - phi) <= 1e-11 * np.linalg.norm(phi)


def test_library_host_weights_are_the_factorial_ratios():
    from paper_1002_3094_gb300.laguerre import laguerre_weights
    for m in range(0, 30):
        a, w = laguerre_weights(m, 5)
        exact = Fraction(math.factorial(m), math.factorial(m + 5))
        assert a * a == pytest.approx(float(exact), rel=1e-13) and w * w == pytest.approx(float(1 / exact), rel=1e-13)


def test_wavelet_coefficients_match_quadrature():
    """Input generator of the chain workload: the trapezoid-rule coefficients
    of the Eq. functiont wavelet against adaptive quadrature with SciPy's
    Laguerre polynomials (Eq. series_lag)."""
    from workloads.laguerre import ALPHA, H_LAG, source_wavelet, wavelet_coefficients
    got = wavelet_coefficients(12)
    for m in (0, 3, 11):
        c = math.sqrt(H_LAG * math.factorial(m) / math.factorial(m + ALPHA))
        g = lambda t: source_wavelet(t) * c * np.exp(-H_LAG * t / 2) * special.eval_genlaguerre(m, ALPHA, H_LAG * t)
        want = integrate.quad(g, 0.0, 0.5, limit=800, points=[0.2], epsabs=1e-30, epsrel=1e-11)[0]
        assert got[m] == pytest.approx(want, rel=1e-6, abs=1e-12 * np.abs(got).max())
