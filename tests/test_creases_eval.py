"""Pins of the crease evaluation (E and p of Sec. 5) on hand-built cases: an
exact reconstruction, one shifted by a known distance, one outside the
neighbourhood, a partial one, and the choice between two candidate chains;
and the joining of marching-squares segments into chains."""
import math

import numpy as np

from paper_1611_06906_gb300 import creases


def _poly(points):
    p = np.asarray(points, dtype=np.float64)
    return np.concatenate([p[:-1], p[1:]], axis=1)


TRUTH = [(10.0, 10.0, 30.0, 10.0), (30.0, 10.0, 30.0, 25.0)]


def test_exact_and_shifted_reconstructions():
    exact = _poly([(10, 10), (20, 10), (30, 10), (30, 18), (30, 25)])
    E, p = creases.evaluate(exact, TRUTH)
    assert E < 1e-12 and p == 1.0
    shifted = _poly([(10, 11.5), (20, 11.5), (30, 11.5)])  # 1.5 px below the first segment only
    E, p = creases.evaluate(shifted, TRUTH[:1])
    assert abs(E - 1.5) < 1e-12 and p == 1.0
    far = _poly([(10, 17.0), (30, 17.0)])  # 7 px away: outside the 6-pixel neighbourhood
    E, p = creases.evaluate(far, TRUTH[:1])
    assert math.isnan(E) and p == 0.0


def test_partial_detection_and_best_chain():
    # only the horizontal segment is found: p is its share of the length (20 of 35)
    E, p = creases.evaluate(_poly([(10, 10), (30, 10)]), TRUTH)
    assert abs(p - 20.0 / 35.0) < 1e-12 and E < 1e-12
    # two chains near the segment: the nearer one (Hausdorff 1) wins over the farther (Hausdorff 3)
    two = np.concatenate([_poly([(10, 13), (30, 13)]), _poly([(10, 9), (30, 9)])])
    E, p = creases.evaluate(two, TRUTH[:1])
    assert abs(E - 1.0) < 1e-12 and p == 1.0


def test_chains_join_at_shared_endpoints():
    s = np.array([[0, 0, 1, 0], [1, 0, 2, 1], [5, 5, 6, 5], [2, 1, 3, 1]], dtype=np.float64)
    groups = sorted(sorted(g.tolist()) for g in creases.chains(s))
    assert groups == [[0, 1, 3], [2]]


def test_replayed_centre_lines_lie_on_the_rendered_vessels():
    """The ground truth of the evaluation: the generator's centre lines, replayed
    from its seed, run through the dark vessels it rendered (noise-free tree:
    the centre of a piece of radius >= 2 lies at least 0.3 below the image 3
    radii away along its normal, except where that point falls on another
    branch near a junction)."""
    from paper_1611_06906_gb300 import synth
    w, h = 200, 160
    img = synth.vessel_tree(77, w, h, depth=4, r0=4.0, noise=0.0).astype(np.float64)
    segs = synth.vessel_tree_centrelines(77, w, h, depth=4, r0=4.0, noise=0.0)
    assert len(segs) == 3 * (2 ** 4 - 1)
    contrast = []
    for ax, ay, bx, by, rad in segs:
        mx, my = 0.5 * (ax + bx), 0.5 * (ay + by)
        x, y = int(round(mx)), int(round(my))
        if rad < 2.0 or not (8 <= x < w - 8 and 8 <= y < h - 8):
            continue
        nx, ny = -(by - ay), bx - ax  # normal of the piece
        n = math.hypot(nx, ny)
        ox, oy = int(round(mx + 3 * rad * nx / n)), int(round(my + 3 * rad * ny / n))
        if not (0 <= ox < w and 0 <= oy < h):
            continue
        contrast.append(img[oy, ox] - img[y, x])
    contrast = np.array(contrast)
    assert contrast.size >= 5 and np.median(contrast) > 0.3 and (contrast > 0.3).mean() >= 0.8
