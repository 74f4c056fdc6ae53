"""Exact 4x4 master equations against oracle histograms (G-tests).

The master equations (oracle/master_eq.py) are written with heights, the
oracle with slope bits; agreement pins Eq. (1)'s slope-bit reading, O1's
uniform site selection and O2's schedule (origin, set permutation, block-level
set draws, acceptance) at thread cells of 2x2 sites.  Negative controls show
that each test can tell the two dynamics apart."""
import numpy as np
import pytest

from oracle import master_eq as me

P_MIN = 1e-4


@pytest.fixture(scope="module")
def space():
    return me.reachable_states()


def _exact_probs(oracle, p, q):
    return oracle.threshold32(p) / 2**32, oracle.threshold32(q) / 2**32


def _histogram(X, Y, index):
    counts = np.zeros(len(index))
    for r in range(X.shape[0]):
        counts[index[me.bits_to_code(X[r], Y[r])]] += 1
    return counts


def test_state_space_is_closed_and_balanced(oracle, space):
    states, index = space
    assert len(states) == 990
    # every reachable configuration is a valid torus height field
    for c in states[::37]:
        X, Y = me.code_to_bits(c)
        assert oracle.invariants(X, Y) == 0
    # height and slope views agree on which sites are extremal
    for c in states[::53]:
        X, Y = me.code_to_bits(c)
        h = me.decode(c)
        for y in range(4):
            for x in range(4):
                assert oracle.site_kind(X, Y, x, y) == me.kind(h, x, y)


def test_symmetric_rates_give_uniform_stationary_state(space):
    states, index = space
    T = me.rs_attempt_matrix(states, index, 0.5, 0.5)
    assert np.allclose(T, T.T)
    u = np.full(len(states), 1.0 / len(states))
    assert np.allclose(u @ T, u)


def test_order_recursion_equals_explicit_permutations(space):
    states, index = space
    a = me.dtrdt_mcs_matrix(states, index, 0.6, 0.3)
    b = me.dtrdt_mcs_matrix_by_orders(states, index, 0.6, 0.3)
    assert np.allclose(a, b, atol=1e-13)


@pytest.mark.parametrize("p,q,n_mcs", [(0.7, 0.2, 1), (0.7, 0.2, 3), (1.0, 0.0, 2)])
def test_sequential_rs_matches_master_equation(oracle, space, p, q, n_mcs):
    states, index = space
    pe, qe = _exact_probs(oracle, p, q)
    T = me.rs_attempt_matrix(states, index, pe, qe)
    pi = me.distribution(T, 16 * n_mcs, len(states))
    X, Y = oracle.seq_rs_many(4, p, q, 1000, 200_000, n_mcs)
    counts = _histogram(X, Y, index)
    G, dof, pval = me.g_test(counts, pi)
    assert pval > P_MIN, (G, dof, pval)


@pytest.mark.parametrize("p,q,n_mcs", [(0.7, 0.2, 1), (0.7, 0.2, 2), (1.0, 0.0, 1)])
def test_dtrdt_matches_master_equation(oracle, space, p, q, n_mcs):
    states, index = space
    pe, qe = _exact_probs(oracle, p, q)
    T = me.dtrdt_mcs_matrix(states, index, pe, qe)
    pi = me.distribution(T, n_mcs, len(states))
    prm = oracle.Params(L=4, p=p, q=q, seed=0, Bx=2, By=2, cx=2, cy=2)
    X, Y = oracle.dtrdt_many(prm, 5000, 200_000, n_mcs)
    counts = _histogram(X, Y, index)
    G, dof, pval = me.g_test(counts, pi)
    assert pval > P_MIN, (G, dof, pval)


def test_tests_discriminate_the_two_dynamics(oracle, space):
    """Negative control: the RS histogram fails against the DTrDT master
    equation and vice versa."""
    states, index = space
    pe, qe = _exact_probs(oracle, 0.7, 0.2)
    pi_rs = me.distribution(me.rs_attempt_matrix(states, index, pe, qe), 16, len(states))
    pi_dd = me.distribution(me.dtrdt_mcs_matrix(states, index, pe, qe), 1, len(states))
    Xs, Ys = oracle.seq_rs_many(4, 0.7, 0.2, 77, 200_000, 1)
    prm = oracle.Params(L=4, p=0.7, q=0.2, seed=0, Bx=2, By=2, cx=2, cy=2)
    Xd, Yd = oracle.dtrdt_many(prm, 88, 200_000, 1)
    assert me.g_test(_histogram(Xs, Ys, index), pi_dd)[2] < 1e-8
    assert me.g_test(_histogram(Xd, Yd, index), pi_rs)[2] < 1e-8
