"""The ARS3 IMEX tableaux the library hands out (fld_ars3_tableau, a host function: no GPU)
against the order conditions of ARS(2,3,3) (Ascher, Ruuth and Spiteri 1997), the scheme
Sect. 3 combines its explicit and implicit terms with, and the third-order convergence of
the resulting IMEX integration of a split linear problem."""
import numpy as np
import pytest


def _tableau():
    from paper_2503_02764_gb300 import fld
    return fld.fld_ars3_tableau()


def test_order_conditions():
    Ae, Ai, b, c = _tableau()
    g = (3 + np.sqrt(3)) / 6
    assert c == pytest.approx([0.0, g, 1 - g], abs=1e-15)
    for A in (Ae, Ai):
        assert A.sum(axis=1) == pytest.approx(c, abs=1e-15)        # stage times
        assert b.sum() == pytest.approx(1.0, abs=1e-15)            # order 1
        assert b @ c == pytest.approx(0.5, abs=1e-15)              # order 2
        assert b @ (c * c) == pytest.approx(1 / 3, abs=1e-15)      # order 3
        assert b @ A @ c == pytest.approx(1 / 6, abs=1e-15)
    # coupling conditions of a third-order IMEX pair (same b and c for both parts)
    assert b @ Ae @ c == pytest.approx(1 / 6, abs=1e-15)
    assert b @ Ai @ c == pytest.approx(1 / 6, abs=1e-15)
    # explicit part strictly lower triangular, implicit part SDIRK with first stage explicit
    assert np.all(np.triu(Ae) == 0)
    assert np.all(np.triu(Ai, 1) == 0) and Ai[0, 0] == 0 and Ai[1, 1] == Ai[2, 2] == g


def _imex_run(Le, Li, y0, T, n):
    Ae, Ai, b, _ = _tableau()
    dt = T / n
    y = y0.copy()
    I = np.eye(len(y0))
    for _ in range(n):
        Y, Fe, Fi = [], [], []
        for s in range(3):
            rhs = y + dt * sum(Ae[s, j] * Fe[j] + Ai[s, j] * Fi[j] for j in range(s))
            Ys = np.linalg.solve(I - dt * Ai[s, s] * Li, rhs)
            Y.append(Ys)
            Fe.append(Le @ Ys)
            Fi.append(Li @ Ys)
        y = y + dt * sum(b[s] * (Fe[s] + Fi[s]) for s in range(3))
    return y


def test_third_order_on_a_split_linear_problem():
    # dy/dt = Le y + Li y, Le a rotation (explicit, like the hyperbolic terms), Li a
    # relaxation (implicit, like the diffusion and exchange); exact solution by expm
    from scipy.linalg import expm
    Le = np.array([[0.0, 1.0], [-1.0, 0.0]])
    Li = np.array([[-2.0, 1.0], [1.0, -3.0]])
    y0 = np.array([1.0, 0.5])
    T = 1.0
    exact = expm(T * (Le + Li)) @ y0
    errs = [np.linalg.norm(_imex_run(Le, Li, y0, T, n) - exact) for n in (20, 40, 80)]
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > 2.8, (errs, rates)
