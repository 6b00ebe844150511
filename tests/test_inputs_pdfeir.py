"""The Pd/Fe/Ir(111) pair list built from the paper's printed tables
(Supplementary Note 4; reading R23): its shells against the printed row
counts and distances, the closure an ordered-pair sum needs, the agreement of
the rows mapped to d and -d (which checks the angular assignment against the
tables themselves), and the Neel form of the nearest-neighbour DMI."""
import collections
import math

import numpy as np

import inputs


def test_table_rows_and_shells():
    tab = inputs.pdfeir_table()
    assert tab.shape == (360, 5)
    pl = inputs.pdfeir_pairs()
    assert len(pl) == 360
    # every printed |r| is the length of its row's triangular shell
    rnn = 0.707107
    counts = collections.Counter(np.round(tab[:, 4], 6))
    assert len(counts) == 35
    lens = collections.Counter()
    for d1, d2, J, D in pl:
        r = rnn * math.sqrt(d1 * d1 + d1 * d2 + d2 * d2)
        key = min(counts, key=lambda x: abs(x - r))
        assert abs(key - r) <= 2e-6 * max(1.0, r)
        lens[key] += 1
    assert lens == counts
    # largest reach and pair count fit the library's limits
    assert max(max(abs(p[0]), abs(p[1])) for p in pl) == 11


def test_closure_and_printed_pairs():
    pl = inputs.pdfeir_pairs()
    by = {(p[0], p[1]): (p[2], p[3]) for p in pl}
    for (d1, d2), (J, D) in by.items():
        J2, D2 = by[(-d1, -d2)]
        assert J2 == J and D2 == tuple(-x for x in D)
    # the rows the assignment puts on d and -d are negatives of each other to
    # the printed precision of the far shells (a wrong assignment would pair
    # rows of different directions)
    tab = inputs.pdfeir_table()
    asg = {(d1, d2): (row, Dx, Dy) for row, d1, d2, Dx, Dy in inputs.pdfeir_assignment()}
    worst = 0.0
    for (d1, d2), (row, Dx, Dy) in asg.items():
        r2, Dx2, Dy2 = asg[(-d1, -d2)]
        worst = max(worst, abs(Dx + Dx2), abs(Dy + Dy2), abs(tab[row, 3] + tab[r2, 3]), abs(tab[row, 0] - tab[r2, 0]))
    assert worst <= 2e-5  # mRy


def test_nearest_neighbour_dmi_is_neel_and_units():
    pl = inputs.pdfeir_pairs()
    nn = [p for p in pl if p[0] ** 2 + p[0] * p[1] + p[1] ** 2 == 1]
    assert len(nn) == 6
    perp, dz = [], []
    for d1, d2, J, D in nn:
        rx, ry = d1 + 0.5 * d2, math.sqrt(3) / 2 * d2
        assert abs(D[0] * rx + D[1] * ry) <= 1e-4  # in-plane D perpendicular to the bond
        perp.append(-ry * D[0] + rx * D[1])      # (z x r_hat) . D
        dz.append(D[2])
        assert J == 0.832467 * inputs.MRY_TO_MEV
    assert max(perp) - min(perp) <= 1e-4 and min(perp) > 0
    # C3v: D_z alternates between the three bond directions and their images
    assert sorted(np.sign(dz)) == [-1, -1, -1, 1, 1, 1]
    assert abs(abs(dz[0]) - 0.020318 * inputs.MRY_TO_MEV) <= 1e-9
