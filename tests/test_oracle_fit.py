"""Pins of the oracle's BFGS driver and error report: a quadratic with a known minimiser, the
Rosenbrock function (textbook minimum), and hand-computed error statistics."""
import numpy as np

from oracle import fit as FIT


def test_bfgs_quadratic_reaches_the_minimiser():
    g = np.random.default_rng(1)
    Q = g.normal(size=(6, 6))
    Q = Q @ Q.T + 6 * np.eye(6)
    b = g.normal(size=6)
    xstar = np.linalg.solve(Q, b)
    f = lambda x: (0.5 * x @ Q @ x - b @ x, Q @ x - b)
    x, L, it = FIT.bfgs(f, np.ones(6), max_iter=200, gtol=1e-9)
    np.testing.assert_allclose(x, xstar, rtol=1e-7, atol=1e-9)
    assert it < 60


def test_bfgs_rosenbrock():
    def f(x):
        a, b = x
        return (1 - a) ** 2 + 100 * (b - a * a) ** 2, np.array([-2 * (1 - a) - 400 * a * (b - a * a), 200 * (b - a * a)])
    x, L, it = FIT.bfgs(f, np.array([-1.2, 1.0]), max_iter=500, gtol=1e-12)
    np.testing.assert_allclose(x, [1.0, 1.0], atol=1e-5)
    assert L < 1e-10


def test_error_report_by_hand():
    off = np.array([0, 2, 5])
    E, Er = np.array([1.0, 3.0]), np.array([0.0, 0.0])          # per atom: 0.5, 1.0
    F = np.zeros((5, 3))
    Fr = np.zeros((5, 3))
    F[0] = [3, 4, 0]                                              # |dF| = 5, others 0
    W = np.zeros((2, 3, 3))
    Wr = np.zeros((2, 3, 3))
    W[1, 0, 1] = -2.0
    r = FIT.errors(E, F, W, Er, Fr, Wr, off)
    np.testing.assert_allclose(r, [1.0, 0.75, np.sqrt((0.25 + 1.0) / 2), 5.0, 1.0, np.sqrt(25 / 5),
                                   2.0, 2.0 / 18, np.sqrt(4.0 / 18)])
