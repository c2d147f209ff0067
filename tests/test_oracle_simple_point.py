"""Pins of the oracle's simple-point (topology) test, Eq. equa:energy1's E_topo term.

The oracle decides "removing block p keeps its superpixel 4-connected" by a breadth-first
search in the 3x3 window.  These tests pin it to (a) the classical digital-topology
definition of a simple point, (b) global connectivity on random windows, (c) hand-checked
spot values."""
import numpy as np
import pytest
import scipy.ndimage as ndi

import oracle

RING = [(-1, -1), (0, -1), (1, -1), (1, 0), (1, 1), (0, 1), (-1, 1), (-1, 0)]  # NW N NE E SE S SW W
S4 = ndi.generate_binary_structure(2, 1)
S8 = ndi.generate_binary_structure(2, 2)


def window(mask):
    g = np.zeros((3, 3), bool)
    for i, (dx, dy) in enumerate(RING):
        if mask >> i & 1:
            g[1 + dy, 1 + dx] = True
    return g


def classical_simple(mask):
    """(4,8) simple point: T4(foreground) == 1 and T8(background) == 1 (Rosenfeld)."""
    fg = window(mask)
    lab, n = ndi.label(fg, S4)
    four = {(0, 1), (1, 2), (2, 1), (1, 0)}
    t4 = len({lab[r, c] for (r, c) in four if lab[r, c] > 0})
    bg = ~fg
    bg[1, 1] = False
    _, t8 = ndi.label(bg, S8)
    return t4 == 1 and t8 == 1


@pytest.fixture(scope="module")
def lut():
    return oracle.simple_lut()


def test_count_and_spot_values(lut):
    assert int(lut.sum()) == 117
    assert lut[0x00] == 0          # no neighbour in the label: removing p would empty it locally
    assert lut[0x0A] == 0          # N and E without NE: they touch only through p
    assert lut[0x0E] == 1          # N, NE, E form one arc
    assert lut[0x22] == 0          # N and S: p is a bridge
    assert lut[0x88] == 0          # E and W: p is a bridge
    assert lut[0xFF] == 1          # interior point
    assert lut[0x02] == 1          # a single 4-neighbour (end of a line)
    assert lut[0x01] == 0          # only a diagonal: not 4-adjacent


def test_matches_classical_definition_except_full_ring(lut):
    diff = [m for m in range(256) if bool(lut[m]) != classical_simple(m)]
    assert diff == [0xFF]
    assert sum(classical_simple(m) for m in range(256)) == 116


def test_window_connectivity_iff(lut):
    """With nothing outside the 3x3 window: for every mask whose window (with p) is one
    4-component, removing p leaves one 4-component iff the mask is simple."""
    checked = 0
    for m in range(1, 256):
        g = window(m)
        g_with = g.copy()
        g_with[1, 1] = True
        if ndi.label(g_with, S4)[1] != 1:
            continue
        after = ndi.label(g, S4)[1]
        assert bool(lut[m]) == (after == 1), hex(m)
        checked += 1
    assert checked > 100


def test_random_windows_removal_keeps_connectivity(lut):
    """Locally simple => globally connected after removal, on random 7x7 foregrounds."""
    rng = np.random.default_rng(0)
    hits = 0
    for _ in range(20000):
        g = rng.random((7, 7)) < 0.6
        g[3, 3] = True
        lab, n = ndi.label(g, S4)
        comp = lab == lab[3, 3]
        m = 0
        for i, (dx, dy) in enumerate(RING):
            if comp[3 + dy, 3 + dx]:
                m |= 1 << i
        if not lut[m]:
            continue
        rest = comp.copy()
        rest[3, 3] = False
        assert rest.any()
        assert ndi.label(rest, S4)[1] == 1
        hits += 1
    assert hits > 1000
