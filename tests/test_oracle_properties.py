"""Property-based pins of the oracle (hypothesis searches small point sets,
shrinking any counterexample): the hull equals brute force, and no filter
rule ever drops an output point.  CPU only; skipped where hypothesis is not
installed."""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

import oracle  # noqa: E402
from oracle import brute  # noqa: E402
from oracle import filter16_ref as G  # noqa: E402
from oracle import filter_ref as F  # noqa: E402

@st.composite
def point_sets(draw, max_n=60):
    # small coordinate ranges force ties, duplicates and collinear runs; some
    # sets use the whole domain
    hi = draw(st.sampled_from([6, 40, (1 << 24) - 1]))
    c = st.integers(0, hi)
    n = draw(st.integers(1, max_n))
    xs = draw(st.lists(c, min_size=n, max_size=n))
    ys = draw(st.lists(c, min_size=n, max_size=n))
    return np.stack([xs, ys], 1).astype(np.float32)


@settings(max_examples=300, deadline=None)
@given(point_sets())
def test_hull_equals_brute_force(pts):
    np.testing.assert_array_equal(oracle.hull(pts), brute.hull(pts))


@settings(max_examples=300, deadline=None)
@given(point_sets())
def test_octagon_and_16gon_filters_keep_every_output_point(pts):
    full = oracle.hull(pts)
    for lab, ext in ((F.labels(pts), F.extremes(pts)), (G.labels16(pts), G.extremes16(pts))):
        kept = lab > 0
        kept[ext] = True
        assert kept[full].all()


@settings(max_examples=300, deadline=None)
@given(point_sets(), st.data())
def test_sampled16_drop_never_drops_an_output_point(pts, data):
    n = pts.shape[0]
    sample = np.array(sorted(data.draw(st.sets(st.integers(0, n - 1), min_size=1, max_size=n))), np.int64)
    drop = G.hull_drop_sampled16(pts, sample)
    assert not drop[oracle.hull(pts)].any()
