"""The seeded target rasterisers: the even-odd polygon fill (per-row crossing
counts) equals a per-sample crossing test written out in plain Python, the
coverage is the 4 x 4 sample mean, and the target families keep unit sum and
odd size."""
import numpy as np

from paper_2512_04556_gb300 import workloads as wl


def _polygon_brute(verts, K):
    """Per supersample point: count the edges that cross its row to its right."""
    h = (K - 1) / 2.0
    axis = [(c - h) + (k - 1.5) / 4.0 for c in range(K) for k in range(4)]
    n = len(verts)
    inside = np.zeros((4 * K, 4 * K), bool)
    for r, y in enumerate(axis):
        for q, x in enumerate(axis):
            odd = False
            for i in range(n):
                x1, y1 = float(verts[i][0]), float(verts[i][1])
                x2, y2 = float(verts[(i + 1) % n][0]), float(verts[(i + 1) % n][1])
                if (y1 > y) != (y2 > y):
                    xint = (x2 - x1) * (y - y1) / (y2 - y1) + x1
                    if x < xint:
                        odd = not odd
            inside[r, q] = odd
    cov = inside.reshape(K, 4, K, 4).mean(axis=(1, 3))
    return cov / cov.sum() if cov.sum() > 0 else None


def test_polygon_fill_matches_per_sample_crossings():
    g = np.random.default_rng(11)
    for t in range(24):
        K = int(g.integers(1, 6)) * 2 + 1
        nv = int(g.integers(3, 10))
        v = g.uniform(-(K - 1) / 2 - 0.5, (K - 1) / 2 + 0.5, (nv, 2))
        if t % 3 == 0:
            v = np.round(v * 4) / 4 - 0.125      # vertices on the sample lattice
        if t % 4 == 0:
            v[1, 1] = v[0, 1]                    # a horizontal edge
        want = _polygon_brute(v, K)
        got = wl.polygon(v, K)
        if want is None:                          # empty polygon: centre impulse
            assert got.sum() == 1.0 and got[(K - 1) // 2, (K - 1) // 2] == 1.0
        else:
            np.testing.assert_array_equal(got, want)


def test_target_families_are_unit_sum_and_odd():
    for t in wl.shape_batch(40) + wl.ring_batch(10) + [wl.disk(3.5), wl.ellipse(9.0, 2.5, 0.7),
                                                       wl.gaussian(2.0), wl.line(9.0)]:
        assert t.shape[0] == t.shape[1] and t.shape[0] % 2 == 1
        assert abs(t.sum() - 1.0) < 1e-12 and t.min() >= 0.0
    # coverage is a count of the pixel's 16 samples: the centre pixel of a
    # radius-2 disk is fully covered, so every pixel is a multiple of it / 16
    d = wl.disk(2.0, 5)
    counts = d / d[2, 2] * 16
    np.testing.assert_allclose(counts, np.round(counts), atol=1e-12)
    assert counts.max() == 16 and counts[0, 0] == 0
