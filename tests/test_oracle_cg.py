"""Pins for the oracle's heat-conduction operator and CG solvers."""
import math

import numpy as np

import oracle
from synth import workloads as W


def test_operator_two_cell_closed_form():
    """2x2 grid with conductivity 1 | 3 per row: the x-face between the cells
    has the harmonic mean 2*1*3/(1+3) = 1.5, boundary faces take the cell's
    own conductivity, the y-face between rows hmean(1,1) = 1 (or 3).
    (A e_00)_00 = 1 + 1 (W) + 1.5 (E) + 1 (S) + 1 (N) = 5.5, (A e_00)_01 = -1.5,
    (A e_00)_10 = -1 (north neighbour)."""
    kappa = np.array([[1.0, 3.0], [1.0, 3.0]])
    e = np.zeros((2, 2))
    e[0, 0] = 1.0
    w = oracle.matvec(kappa, e)
    assert w[0, 0] == 5.5
    assert w[0, 1] == -1.5
    assert w[1, 0] == -1.0
    assert w[1, 1] == 0.0
    e = np.zeros((2, 2))
    e[1, 1] = 1.0
    w = oracle.matvec(kappa, e)
    assert w[1, 1] == 1 + 1.5 + 3 + 3 + 3
    assert w[1, 0] == -1.5 and w[0, 1] == -3.0


def _eigvec(n, p, q):
    i = np.arange(n)
    sx = np.sin(np.pi * p * (i + 1) / (n + 1))
    sy = np.sin(np.pi * q * (i + 1) / (n + 1))
    return np.outer(sy, sx)


def test_operator_eigenmode_constant_conductivity():
    """Constant kappa: A = I + kappa * (-L_Dirichlet), so sin modes are
    eigenvectors with mu = 1 + kappa (4 sin^2(pi p/(2(n+1))) + 4 sin^2(pi q/(2(n+1))))."""
    n, kap = 23, 2.5
    for p, q in [(1, 1), (3, 5), (7, 2)]:
        u = _eigvec(n, p, q)
        mu = 1 + kap * (4 * math.sin(math.pi * p / (2 * (n + 1))) ** 2 + 4 * math.sin(math.pi * q / (2 * (n + 1))) ** 2)
        w = oracle.matvec(np.full((n, n), kap), u)
        assert np.abs(w - mu * u).max() < 1e-13 * mu


def test_operator_symmetric_positive_definite():
    n = 9
    kappa, _ = W.cg_problem(n, 1e-2, 1e2)
    A = np.zeros((n * n, n * n))
    for k in range(n * n):
        e = np.zeros(n * n)
        e[k] = 1.0
        A[:, k] = oracle.matvec(kappa, e.reshape(n, n)).ravel()
    assert np.abs(A - A.T).max() <= 1e-12 * np.abs(A).max()
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() >= 1.0 - 1e-12


def test_cg64_eigenmode_one_iteration():
    """With an eigenvector right-hand side, CG converges in one step to b/mu."""
    n, kap, p, q = 31, 0.7, 2, 3
    b = _eigvec(n, p, q)
    mu = 1 + kap * (4 * math.sin(math.pi * p / (2 * (n + 1))) ** 2 + 4 * math.sin(math.pi * q / (2 * (n + 1))) ** 2)
    x, it, rr = oracle.cg64(np.full((n, n), kap), b, tol=1e-10)
    assert it == 1
    assert np.abs(x - b / mu).max() < 1e-14


def test_cg64_against_dense_solve():
    n = 14
    kappa, b = W.cg_problem(n, 1e-2, 1e2)
    A = np.zeros((n * n, n * n))
    for k in range(n * n):
        e = np.zeros(n * n)
        e[k] = 1.0
        A[:, k] = oracle.matvec(kappa, e.reshape(n, n)).ravel()
    xd = np.linalg.solve(A, b.ravel()).reshape(n, n)
    x, it, rr = oracle.cg64(kappa, b, tol=1e-13)
    assert rr <= 1e-13
    assert np.abs(x - xd).max() <= 1e-10 * np.abs(xd).max()
    assert oracle.relres(kappa, b, x) <= 1e-12


def test_refinement_reaches_tolerance_and_matches_fp64():
    n = 40
    kappa, b = W.cg_problem(n, 1e-1, 1e1)
    x64, it64, _ = oracle.cg64(kappa, b, tol=1e-12)
    xr, it, rel, outer = oracle.cg_refine(kappa, b, tol=1e-10, inner_tol=1e-4)
    assert rel <= 1e-10 and outer >= 2
    assert oracle.relres(kappa, b, xr) <= 1e-10
    assert np.abs(xr - x64).max() <= 1e-8 * np.abs(x64).max()


def test_refinement_inner_cg_eigenmode_one_iteration():
    """The FP32 inner CG on an eigenvector right-hand side: its Krylov space
    has one dimension, so with the right step length the first inner solve
    ends after one iteration with an FP32-rounding-level residual (about
    1e-7 relative), and one correction already meets a 1e-6 tolerance.  A
    wrong step length (or a wrong dot product in it) leaves a residual near
    the right-hand side's size and needs many more iterations."""
    n, kap, p, q = 31, 0.7, 2, 3
    b = _eigvec(n, p, q)
    xr, it, rel, outer = oracle.cg_refine(np.full((n, n), kap), b, tol=1e-6, inner_tol=1e-4)
    assert it == 1 and outer == 1
    assert 1e-9 < rel <= 1e-6  # an FP32 solve: rounding level, not an FP64 one
    mu = 1 + kap * (4 * math.sin(math.pi * p / (2 * (n + 1))) ** 2 + 4 * math.sin(math.pi * q / (2 * (n + 1))) ** 2)
    assert np.abs(xr - b / mu).max() <= 1e-6 * np.abs(b / mu).max()
