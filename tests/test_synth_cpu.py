"""Seeded input generators: the city-block workload (12 uneven sub-regions,
20M Gaussians, 6 views each) keeps its stated sizes and is reproducible."""
import numpy as np

import pgsag_synth as syn


def test_config4_sizes_follow_uneven_pattern():
    s = syn.config4_sizes()
    assert len(s) == 12 and sum(s) == 20_000_000
    assert all(b > a for a, b in zip(s, s[1:]))
    # the config-3 pattern's spread (3M / 200k = 15) is kept
    assert 14.0 < s[-1] / s[0] < 16.0


def test_config4_small_scale_views_and_lazy_images():
    g, ranges, cams, owner, masks, targets = syn.config4(scale=0.001)
    assert len(cams) == 72 and len(masks) == 72 and len(targets) == 72
    assert owner == [r for r in range(12) for _ in range(6)]
    assert ranges[0][0] == 0 and ranges[-1][1] == g.n
    assert all(b0 == a1 for (_, a1), (b0, _) in zip(ranges, ranges[1:]))
    c = cams[0]
    assert (c.width, c.height) == (int(6000 * 0.001 ** 0.5), int(4000 * 0.001 ** 0.5))
    assert abs(c.fx - 1.2 * c.width) < 1e-3
    for v in (0, 17, 71):
        m = masks[v]
        assert m.shape == (c.height, c.width) and m.dtype == np.uint8
        assert 0.17 <= m.mean() <= 0.63
        assert np.array_equal(m, masks[v])          # per-view seed: same image on every access
        t = targets[v]
        assert t.shape == (c.height, c.width, 3) and np.array_equal(t, targets[v])
    assert not np.array_equal(targets[0], targets[1])
