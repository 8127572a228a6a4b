"""The union-bound tool: its distance-spectrum walk against the textbook
spectra of tests/golden/distance_spectra.txt, and the bound's basic shape.
CPU only."""
import math
import os

import pytest

from paper_2011_09337_gb300 import ber

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "distance_spectra.txt")


def _rows():
    with open(GOLDEN) as fh:
        return [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]


@pytest.mark.parametrize("key", sorted({" ".join(r[:3]) for r in _rows()}))
def test_spectrum_matches_textbook(key):
    rows = [r for r in _rows() if " ".join(r[:3]) == key]
    K, beta = int(rows[0][0]), int(rows[0][1])
    polys = tuple(int(p, 8) for p in rows[0][2].split(","))
    spec = ber.distance_spectrum(K, beta, polys, max(int(r[3]) for r in rows))
    assert min(spec) == int(rows[0][3])  # free distance
    for r in rows:
        d, ad, cd = int(r[3]), int(r[4]), int(r[5])
        if ad >= 0:
            assert spec[d][0] == ad
        if cd >= 0:
            assert spec[d][1] == cd


def test_union_bound_shape():
    K, beta, polys = 7, 2, (0o171, 0o133)
    vals = [ber.union_bound(K, beta, polys, e) for e in (2.0, 3.0, 4.0, 5.0, 6.0)]
    assert all(a > b for a, b in zip(vals, vals[1:]))
    # at high Eb/N0 the free-distance term dominates: 36 Q(sqrt(2 * 10 * R * Eb/N0))
    g = 10 ** 0.6
    lead = 36 * 0.5 * math.erfc(math.sqrt(2 * 10 * 0.5 * g) / math.sqrt(2))
    assert 0.85 * vals[-1] < lead <= vals[-1]


def test_catastrophic_code_is_refused():
    # K=3 generators 110 and 011 share the factor 1 + D: a weight-0 cycle
    with pytest.raises(ValueError):
        ber.distance_spectrum(3, 2, (0o6, 0o3), 12)
