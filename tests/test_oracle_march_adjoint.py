"""Pins of the oracle's march derivatives (fixed local time step).

The march with a given dt is checked against the oracle's own march with
its frozen dt (pinned in test_oracle_pins.py); the reverse sweep of the
march against central finite differences of J = g . q_N (an independent
fact: only forward marches are differenced) and against the tangent march
by the dot-product identity <g, dq_N> = <qbar_0, dq_0> + <nbar, dn> (two
separately written sweeps: the tangent follows the stages forward, the
reverse runs them backward from stored stage states).  CPU only.
"""
import numpy as np
import pytest

import oracle
from paper_1403_7209_gb300 import meshgen


def setup(n, seed):
    m = meshgen.lattice(n, seed=seed)
    q = meshgen.flow_state(m, seed=seed)
    lam = oracle.spectral_radius(m.edge, q, m.normal)
    dt = oracle.time_step(m.volume, lam, 0.5)
    return m, q, dt


@pytest.mark.parametrize("order", [1, 2])
def test_fixed_dt_march_equals_the_march(order):
    m, q, dt = setup(4, 0)
    qa, sa = oracle.march(order, 3, m.edge, q, m.normal, m.dx, m.volume)
    qb, sb = oracle.march_dt(order, 3, m.edge, q, m.normal, m.dx, m.volume, dt)
    assert sa == sb == 0
    np.testing.assert_array_equal(qa, qb)


@pytest.mark.parametrize("order", [1, 2])
def test_dot_product_tangent_vs_reverse(order):
    m, q, dt = setup(4, 1)
    rng = np.random.default_rng(order)
    g = rng.normal(size=q.shape)
    qd = rng.normal(size=q.shape)
    nd = rng.normal(size=m.normal.shape)
    _, qdN = oracle.march_tangent(order, 3, m.edge, q, m.normal, m.dx, m.volume, dt, qd, nd)
    qb, nb = oracle.march_reverse(order, 3, m.edge, q, m.normal, m.dx, m.volume, dt, g)
    lhs = float(np.sum(g * qdN))
    rhs = float(np.sum(qb * qd) + np.sum(nb * nd))
    assert abs(lhs - rhs) <= 1e-12 * (np.sum(np.abs(g * qdN)) + np.sum(np.abs(qb * qd)))


@pytest.mark.parametrize("order", [1, 2])
def test_reverse_matches_central_differences(order):
    # n = 3, 2 steps: every stage state's kink margin (|u.n| and the wave
    # speed gap of each face) is far above the perturbation (h = 1e-8 in q
    # or n moves the stage states by ~1e-7), so J is smooth on [-h, h]
    m, q, dt = setup(3, 0)
    steps, h = 2, 1e-8
    rng = np.random.default_rng(10 + order)
    g = rng.normal(size=q.shape)
    qb, nb, S = oracle.march_reverse(order, steps, m.edge, q, m.normal, m.dx, m.volume, dt, g,
                                     with_states=True)
    margin = min(oracle.kink_margin(order, m.edge, s, m.normal, m.dx, m.volume).min() for s in S)
    assert margin > 1000 * h

    def J(qq, nn):
        qN, st = oracle.march_dt(order, steps, m.edge, qq, nn, m.dx, m.volume, dt)
        assert st == 0
        return float(np.sum(g * qN))

    for _ in range(3):
        v = rng.normal(size=q.shape)
        fd = (J(q + h * v, m.normal) - J(q - h * v, m.normal)) / (2 * h)
        assert fd == pytest.approx(float(np.sum(qb * v)), rel=1e-6)
        w = rng.normal(size=m.normal.shape)
        fd = (J(q, m.normal + h * w) - J(q, m.normal - h * w)) / (2 * h)
        assert fd == pytest.approx(float(np.sum(nb * w)), rel=1e-6)


def test_one_stage_reduces_to_the_residual_reverse():
    # one forward-Euler stage q1 = q - D R(q): qbar = g + dR/dq^T (-D g)
    m, q, dt = setup(4, 2)
    g = np.random.default_rng(3).normal(size=q.shape)
    qb, nb = oracle.march_reverse(2, 1, m.edge, q, m.normal, m.dx, m.volume, dt, g, stages=1)
    lam = -(dt / m.volume)[:, None] * g
    rb, rn = oracle.residual_reverse(2, m.edge, q, m.normal, m.dx, m.volume, lam)
    np.testing.assert_allclose(qb, rb + g, rtol=1e-15, atol=1e-300)
    np.testing.assert_array_equal(nb, rn)


def test_zero_steps_and_linearity_in_g():
    m, q, dt = setup(4, 3)
    rng = np.random.default_rng(4)
    g1, g2 = rng.normal(size=q.shape), rng.normal(size=q.shape)
    qb, nb = oracle.march_reverse(2, 0, m.edge, q, m.normal, m.dx, m.volume, dt, g1)
    np.testing.assert_array_equal(qb, g1)
    assert np.all(nb == 0.0)
    a1, n1 = oracle.march_reverse(2, 2, m.edge, q, m.normal, m.dx, m.volume, dt, g1)
    a2, n2 = oracle.march_reverse(2, 2, m.edge, q, m.normal, m.dx, m.volume, dt, g2)
    a3, n3 = oracle.march_reverse(2, 2, m.edge, q, m.normal, m.dx, m.volume, dt, 2 * g1 + g2)
    np.testing.assert_allclose(a3, 2 * a1 + a2, rtol=1e-12, atol=1e-12 * np.abs(a3).max())
    np.testing.assert_allclose(n3, 2 * n1 + n2, rtol=1e-12, atol=1e-12 * np.abs(n3).max())
