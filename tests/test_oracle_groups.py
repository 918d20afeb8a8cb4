"""Pins of the oracle's encounter groups (paper Sec. 2: one Bulirsch-Stoer call
over the bodies in encounters; read here as one call per big group and one
per flagged planetesimal, with the planetesimal's group holding the whole big
groups of the bigs it meets and writing back only the planetesimal).

The expected memberships are written out by hand from that reading, so a
one-line slip in the oracle's group construction fails one of them: a union
without path lookup, a group of only the met bigs instead of their whole big
groups, a planetesimal's group that writes back its big members, duplicated
members, or a planetesimal that joins the big groups.  The last test checks
the grouped hybrid step against a brute-force N-body integration (scipy's
DOP853) for a bound pair of giants with a planetesimal in encounter with it.
"""
import numpy as np
import pytest

import oracle as orc
from paper_2601_16791_gb300 import workloads as W

from test_oracle_pins import _nbody_rhs

MU0 = W.G


def groups(nbig, nsmall, pairs):
    return orc.build_groups(nbig, nsmall, pairs)


def test_no_pairs_no_groups():
    assert groups(3, 5, []) == []


def test_single_big_pair_is_one_group_written_whole():
    assert groups(3, 2, [(0, 2)]) == [([0, 2], 0)]


@pytest.mark.parametrize("pairs", [[(0, 1), (1, 2)], [(0, 2), (1, 2)], [(0, 1), (0, 2)],
                                   [(1, 2), (0, 2)], [(0, 2), (1, 2), (0, 1)]])
def test_chain_of_three_bigs_is_one_group(pairs):
    """0-1-2 connected through flagged pairs in any order: one big group; the
    fourth big body meets nothing and has no group."""
    assert groups(4, 3, pairs) == [([0, 1, 2], 0)]


def test_two_disjoint_big_pairs_are_two_groups():
    assert groups(5, 1, [(0, 1), (2, 3)]) == [([0, 1], 0), ([2, 3], 0)]
    # interleaved indices: {0, 3} and {1, 4}
    assert groups(5, 1, [(0, 3), (1, 4)]) == [([0, 3], 0), ([1, 4], 0)]


def test_planetesimal_takes_whole_big_groups_and_writes_only_itself():
    """Planetesimal 6 (index nbig + 1) meets big 1 (group {0, 1}) and big 3
    (group {2, 3}): its group is both whole big groups, bigs ascending, then
    itself; only the last member is written.  The big groups stay separate
    (a massless body joins nothing)."""
    nbig = 5
    got = groups(nbig, 3, [(0, 1), (2, 3), (1, 6), (3, 6)])
    assert got == [([0, 1], 0), ([2, 3], 0), ([0, 1, 2, 3, 6], 4)]


def test_planetesimal_with_a_big_outside_any_big_group():
    """Big 4 is in no flagged big-big pair: the planetesimal's group is big 4
    and itself, and big 4 gets no group of its own."""
    assert groups(5, 2, [(4, 5)]) == [([4, 5], 1)]
    # with a big group elsewhere, it is not pulled in
    assert groups(5, 2, [(0, 1), (4, 5)]) == [([0, 1], 0), ([4, 5], 1)]


def test_planetesimal_meeting_two_bigs_of_one_group_lists_them_once():
    """Planetesimal 5 meets bigs 0 and 2, both in the group {0, 1, 2}: the
    group's three bigs once each, plus the planetesimal; big 1, which it does
    not meet, is in it too."""
    got = groups(4, 2, [(0, 1), (0, 5), (1, 2), (2, 5)])
    assert got == [([0, 1, 2], 0), ([0, 1, 2, 5], 3)]


def test_planetesimals_each_get_their_own_group_in_index_order():
    """Two planetesimals meeting the same big are two groups; a planetesimal
    that meets only a lone big and one that meets a big group differ."""
    got = groups(3, 4, [(0, 1), (0, 6), (0, 4), (2, 5)])
    assert got == [([0, 1], 0), ([0, 1, 4], 2), ([2, 5], 1), ([0, 1, 6], 2)]


def test_pair_validation():
    with pytest.raises(orc.OracleError):
        groups(2, 2, [(2, 3)])      # first index must be a big body
    with pytest.raises(orc.OracleError):
        groups(2, 2, [(1, 1)])      # j > i


def _bound_pair_and_planetesimal(d_ab=0.15, d_p=0.4):
    """Jupiter at 5.2 AU with a 0.1 Jupiter-mass companion on a circular
    orbit 0.15 AU from it (0.42 Hill radii, bound), and a planetesimal on a
    circular heliocentric orbit trailing them by 0.4 AU: inside Jupiter's
    changeover zone from the start."""
    m_a, m_b = W.M_JUP, 0.1 * W.M_JUP
    xa = W.elements_to_xv(MU0 + W.G * m_a, 5.2, 0.0, 0.0, 0.0, 0.0, 0.0)
    xb = xa.copy()
    xb[0] += d_ab
    xb[4] += np.sqrt(W.G * (m_a + m_b) / d_ab)
    xp = W.elements_to_xv(MU0, 5.2, 0.0, 0.0, 0.0, 0.0, -d_p / 5.2)
    return np.array([m_a, m_b]), np.stack([xa, xb, xp], axis=1)


def test_bound_pair_with_planetesimal_vs_brute_force():
    """The pair is flagged at every step (a big group integrated by BS), and
    so is the planetesimal with both bigs (a test-particle group holding the
    big group).  Against DOP853 of the full three-body problem about the
    star over 400 one-day steps, every body stays within 2e-9 (bigs) and
    5e-8 (planetesimal) relative.  Integrating the pair outside BS (only the
    kick's K share of their mutual force) misses by more than 1e-2."""
    from scipy.integrate import solve_ivp
    m_big, xv_helio = _bound_pair_and_planetesimal()
    h, nsteps = 1.0, 400
    p = orc.make_params(W.default_params(h))
    xv, mu, rc = orc.init(p, 2, 1, m_big, xv_helio)
    out, ever, log, st = orc.step(p, 2, xv, mu, rc, None, None, nsteps, log_cap=4 * nsteps)
    pairs = {(int(i), int(j)) for _, i, j in log}
    assert pairs == {(0, 1), (0, 2), (1, 2)}
    assert (log[:, 1:] == [0, 1]).all(axis=1).sum() == nsteps      # pair flagged every step
    hel = orc.readout(p, 2, 1, mu, out)
    mus = np.array([W.G * m_big[0], W.G * m_big[1], 0.0])
    y0 = np.concatenate([xv_helio[:3].ravel(), xv_helio[3:].ravel()])
    sol = solve_ivp(_nbody_rhs(MU0, mus), (0, nsteps * h), y0, method="DOP853",
                    rtol=1e-13, atol=1e-15)
    ref = sol.y[:9, -1].reshape(3, 3)
    err = np.linalg.norm(hel[:3] - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert err[:2].max() < 2e-9, err
    assert err[2] < 5e-8, err
