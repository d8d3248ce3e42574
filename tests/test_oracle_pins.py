"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here calls the CUDA library. Each check derives its expected value
independently of the oracle's code: the ring is rebuilt from the circle's
definition, scores from a brute-force scan over thresholds, pyramid values
from exact area integrals, bins from rational arithmetic, and the Eq. 1
properties from the definition of the union.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle

# --------------------------------------------------------------------------
# independent restatements used as expected values


def ring_from_circle():
    """The 16 pixels of the radius-3 Bresenham circle (Sec. 2), as the points
    whose distance rounds to 3, in angular order starting straight up and
    turning clockwise in image coordinates (y down)."""
    pts = [(dx, dy) for dx in range(-3, 4) for dy in range(-3, 4)
           if round(math.hypot(dx, dy)) == 3]
    assert len(pts) == 16
    # angle measured clockwise from "up" (0, -1)
    return sorted(pts, key=lambda p: math.atan2(p[0], -p[1]) % (2 * math.pi))


RING = ring_from_circle()


def seg_test(img, x, y, t, n=9):
    """Sec. 2: p is a corner iff n contiguous ring pixels are all > I_p + t
    or all < I_p - t."""
    Ip = int(img[y, x])
    v = [int(img[y + dy, x + dx]) for dx, dy in RING]
    for j in range(16):
        arc = [v[(j + m) % 16] for m in range(n)]
        if all(a > Ip + t for a in arc) or all(a < Ip - t for a in arc):
            return True
    return False


def brute_score(img, x, y):
    """Largest t >= 0 for which the segment test fires, 0 if none or if the
    ring leaves the image."""
    h, w = img.shape
    if x < 3 or y < 3 or x >= w - 3 or y >= h - 3:
        return 0
    best = 0
    for t in range(0, 256):
        if seg_test(img, x, y, t):
            best = t
        else:
            break  # the test is monotone in t
    return best


def brute_detect(img, t):
    """Threshold + strict 3x3 non-maximum suppression on brute-force scores."""
    h, w = img.shape
    sc = np.zeros((h, w), int)
    for y in range(h):
        for x in range(w):
            sc[y, x] = brute_score(img, x, y)
    out = []
    for y in range(h):
        for x in range(w):
            v = sc[y, x]
            if v < t:
                continue
            nb = [sc[y + dy, x + dx] if 0 <= y + dy < h and 0 <= x + dx < w else 0
                  for dy in (-1, 0, 1) for dx in (-1, 0, 1) if (dx, dy) != (0, 0)]
            if all(v > q for q in nb):
                out.append((x, y, v))
    return out


def kp_tuples(kp):
    return [(int(k["layer"]), int(k["y"]), int(k["x"]), int(k["score"]), int(k["flags"])) for k in kp]


# --------------------------------------------------------------------------
# segment test and score


def test_ring_is_the_bresenham_circle_in_order():
    # consecutive ring pixels are 8-neighbours, and the ring closes
    for k in range(16):
        a, b = RING[k], RING[(k + 1) % 16]
        assert max(abs(a[0] - b[0]), abs(a[1] - b[1])) == 1
    assert RING[0] == (0, -3) and RING[4] == (3, 0) and RING[8] == (0, 3) and RING[12] == (-3, 0)


def test_score_equals_bruteforce_threshold_scan_random_patches():
    rng = np.random.default_rng(7)
    for trial in range(400):
        kind = trial % 4
        if kind == 0:
            img = rng.integers(0, 256, (7, 7), dtype=np.uint8)
        elif kind == 1:  # low contrast around a mid value
            img = np.clip(128 + rng.integers(-40, 41, (7, 7)), 0, 255).astype(np.uint8)
        elif kind == 2:  # two-level patterns: corners of every shape
            lo, hi = sorted(rng.integers(0, 256, 2))
            img = np.where(rng.random((7, 7)) < 0.5, lo, hi).astype(np.uint8)
        else:  # saturated extremes
            img = rng.choice(np.array([0, 1, 254, 255], np.uint8), (7, 7))
        assert oracle.score(img, 3, 3) == brute_score(img, 3, 3), img


def test_score_all_two_level_ring_patterns():
    """Every one of the 2^16 bright/dark ring patterns: the score is delta-1
    exactly when the pattern has 9 contiguous equal bits (cyclically)."""
    rng = np.random.default_rng(3)
    canvas = np.zeros((7, 7), np.uint8)
    for pattern in range(1 << 16):
        delta = int(rng.integers(1, 128))
        c = 128
        canvas[:] = c
        bits = [(pattern >> k) & 1 for k in range(16)]
        for k, (dx, dy) in enumerate(RING):
            canvas[3 + dy, 3 + dx] = c + delta if bits[k] else c - delta
        run = any(all(bits[(j + m) % 16] == b for m in range(9)) for j in range(16) for b in (0, 1))
        expect = delta - 1 if run else 0
        assert oracle.score(canvas, 3, 3) == expect, (pattern, delta)


def test_score_border_and_constant():
    img = np.full((12, 12), 77, np.uint8)
    assert not oracle.score_image(img).any()
    rng = np.random.default_rng(1)
    img = rng.integers(0, 256, (12, 12), dtype=np.uint8)
    sc = oracle.score_image(img)
    assert not sc[:3].any() and not sc[-3:].any() and not sc[:, :3].any() and not sc[:, -3:].any()


@pytest.mark.parametrize("v", [1, 2, 20, 21, 22, 100, 127])
@pytest.mark.parametrize("sign", [1, -1])
def test_isolated_pixel_gives_one_keypoint(v, sign):
    """A single pixel of contrast v on a flat field: its ring is uniformly
    darker (brighter) by v, so its score is v - 1; every other pixel sees it
    at most once on its ring and scores 0. One keypoint iff v - 1 >= t."""
    t = 20
    img = np.full((40, 48), 128, np.uint8)
    img[17, 23] = 128 + sign * v
    s = oracle.Stream(48, 40, N_r=2, N_c=2, O=1, t=t, mask_mode=oracle.MASK_FULL)
    s.push(img)
    kp = s.keypoints()
    if v - 1 >= t:
        assert kp_tuples(kp) == [(0, 17, 23, v - 1, 0)]
    else:
        assert len(kp) == 0


def test_full_detection_equals_bruteforce_on_tiny_images():
    rng = np.random.default_rng(11)
    for trial in range(6):
        h, w = 14 + trial, 16 + 2 * trial
        base = rng.integers(0, 256, (h, w)).astype(np.float64)
        if trial % 2:
            base = np.round(base / 64) * 64  # blocky: plateaus and corners
        img = np.clip(base, 0, 255).astype(np.uint8)
        t = [5, 20, 40][trial % 3]
        s = oracle.Stream(w, h, N_r=1, N_c=1, O=1, t=t, mask_mode=oracle.MASK_FULL)
        s.push(img)
        got = [(int(k["x"]), int(k["y"]), int(k["score"])) for k in s.keypoints()]
        exp = sorted(brute_detect(img, t), key=lambda p: (p[1], p[0]))
        assert got == exp


def test_nms_ties_suppress_both():
    """Strict maxima: two equal adjacent scores suppress each other."""
    img = np.full((20, 20), 100, np.uint8)
    img[9, 9] = img[9, 10] = 200  # a 2-pixel blob: both see the same arc
    sc = oracle.score_image(img)
    assert sc[9, 9] == sc[9, 10] > 20
    s = oracle.Stream(20, 20, N_r=1, N_c=1, O=1, t=20, mask_mode=oracle.MASK_FULL)
    s.push(img)
    assert len(s.keypoints()) == 0


# --------------------------------------------------------------------------
# pyramid


def area_mean(img, x0, y0, size):
    """Exact mean of the piecewise-constant image over the square
    [x0, x0+size) x [y0, y0+size) (Fractions)."""
    total = Fraction(0)
    h, w = img.shape
    for y in range(h):
        oy = max(Fraction(0), min(Fraction(y + 1), y0 + size) - max(Fraction(y), y0))
        if oy == 0:
            continue
        for x in range(w):
            ox = max(Fraction(0), min(Fraction(x + 1), x0 + size) - max(Fraction(x), x0))
            if ox:
                total += ox * oy * int(img[y, x])
    return total / (size * size)


def round_half_up(q: Fraction) -> int:
    return math.floor(q + Fraction(1, 2))


def test_pyramid_matches_exact_area_means():
    rng = np.random.default_rng(5)
    img = rng.integers(0, 256, (12, 18), dtype=np.uint8)
    layers = oracle.pyramid(img, 2, 1)  # c0, d0, c1, d1
    c0, d0, c1, d1 = layers
    assert (c0 == img).all()
    assert c1.shape == (6, 9) and d0.shape == (8, 12) and d1.shape == (4, 6)
    for y in range(6):
        for x in range(9):
            assert c1[y, x] == round_half_up(area_mean(img, 2 * x, 2 * y, 2))
    for y in range(8):
        for x in range(12):
            q = area_mean(img, Fraction(3, 2) * x, Fraction(3, 2) * y, Fraction(3, 2))
            assert d0[y, x] == round_half_up(q), (x, y)
    for y in range(4):
        for x in range(6):
            assert d1[y, x] == round_half_up(area_mean(d0, 2 * x, 2 * y, 2))


def test_pyramid_geometry_at_paper_scale():
    # 640x480 with 4 octaves + intra-octaves: scales 1, 1.5, 2, 3, 4, 6, 8, 12
    exp = [(640, 480, 2), (426, 320, 3), (320, 240, 4), (213, 160, 6),
           (160, 120, 8), (106, 80, 12), (80, 60, 16), (53, 40, 24)]
    assert [oracle.layer_geom(640, 480, 4, 1, l) for l in range(8)] == exp
    assert oracle.layer_geom(320, 240, 1, 0, 0) == (320, 240, 2)
    assert oracle.num_layers(1, 0) == 1 and oracle.num_layers(5, 1) == 10


def test_pyramid_constant_stays_constant():
    img = np.full((48, 72), 201, np.uint8)
    for layer in oracle.pyramid(img, 3, 1):
        assert (layer == 201).all()


# --------------------------------------------------------------------------
# rotation symmetry of the whole detector


@pytest.mark.parametrize("O,intra,N", [(1, 0, 48), (2, 1, 48), (4, 1, 96)])
def test_rotation_by_90_degrees(O, intra, N):
    """On an N x N frame whose every layer is exact (N divisible by
    3 * 2^(O-1)), rotating the frame rotates every layer's keypoints: the ring
    maps to itself under a quarter turn, the box filters are symmetric and the
    suppression is strict."""
    rng = np.random.default_rng(O * 10 + N)
    img = gaussian_blocks(rng, N)
    def run(im):
        s = oracle.Stream(N, N, N_r=1, N_c=1, O=O, intra=intra, t=15, mask_mode=oracle.MASK_FULL)
        s.push(im)
        return s.keypoints()
    kp = run(img)
    kr = run(np.ascontiguousarray(np.rot90(img)))
    assert len(kp) > 0
    sizes = [oracle.layer_geom(N, N, O, intra, l)[0] for l in range(oracle.num_layers(O, intra))]
    # np.rot90 (counter-clockwise): pixel (x, y) of an n x n layer goes to (y, n-1-x)
    mapped = sorted((int(k["layer"]), sizes[k["layer"]] - 1 - int(k["x"]), int(k["y"]), int(k["score"]))
                    for k in kp)
    got = sorted((int(k["layer"]), int(k["y"]), int(k["x"]), int(k["score"])) for k in kr)
    assert got == mapped


def gaussian_blocks(rng, N):
    img = np.full((N, N), 120.0)
    for _ in range(25):
        x, y = rng.integers(0, N, 2)
        w, h = rng.integers(3, N // 3, 2)
        img[y:y + h, x:x + w] = rng.integers(0, 256)
    img += rng.normal(0, 6, img.shape)
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


# --------------------------------------------------------------------------
# bins (Eq. 3) and masks (Eqs. 2, 4)


def test_block_of_matches_rational_bins():
    """Bin (floor(Y/S_y), floor(X/S_x)) with S_x = W/N_c, S_y = H/N_r exact."""
    rng = np.random.default_rng(2)
    for _ in range(3000):
        W, H = int(rng.integers(8, 700)), int(rng.integers(8, 500))
        N_c, N_r = int(rng.integers(1, min(W, 20) + 1)), int(rng.integers(1, min(H, 20) + 1))
        S = int(rng.choice([2, 3, 4, 6, 8, 12]))
        # a layer pixel whose image position lies inside the frame
        x = int(rng.integers(0, max(1, (2 * W) // S)))
        y = int(rng.integers(0, max(1, (2 * H) // S)))
        X, Y = (x * S) // 2, (y * S) // 2
        if X >= W or Y >= H:
            continue
        c = math.floor(Fraction(X) / Fraction(W, N_c))
        r = math.floor(Fraction(Y) / Fraction(H, N_r))
        assert oracle.block_of(x, y, S, W, H, N_r, N_c) == r * N_c + c


def test_block_edges_hand_placed():
    # 640 x 480, 16 columns x 12 rows: 40 x 40 bins
    assert oracle.block_of(39, 0, 2, 640, 480, 12, 16) == 0
    assert oracle.block_of(40, 0, 2, 640, 480, 12, 16) == 1
    assert oracle.block_of(0, 40, 2, 640, 480, 12, 16) == 16
    # d0 (S = 3): x = 27 sits at X = 40
    assert oracle.block_of(26, 0, 3, 640, 480, 12, 16) == 0
    assert oracle.block_of(27, 0, 3, 640, 480, 12, 16) == 1
    # W = 100, 3 columns: S_x = 33.33, X = 33 -> 0, X = 34 -> 1, X = 67 -> 2
    assert [oracle.block_of(X, 0, 2, 100, 10, 1, 3) for X in (33, 34, 66, 67)] == [0, 1, 1, 2]


def test_intensity_difference_mask_threshold_is_strict():
    """Eq. 2 in the 'detect where it changed' reading, block mean > T_I:
    a block raised by exactly T_I stays inactive, by T_I + 1 turns active."""
    W, H = 64, 48
    f0 = np.full((H, W), 100, np.uint8)
    f1 = f0.copy()
    f1[0:16, 0:16] += 5   # block (0,0): mean |d| = 5 > 4
    f1[16:32, 16:32] += 4  # block (1,1): mean |d| = 4, not > 4
    f1[32:48, 48:64] -= 6  # block (2,3): darker by 6
    s = oracle.Stream(W, H, N_r=3, N_c=4, O=1, T_I=4, t=20, mask_mode=oracle.MASK_ID)
    s.push(f0)
    assert (s.mask() == 1).all()  # first frame: detect everywhere
    s.push(f1)
    exp = np.zeros((3, 4), np.uint8)
    exp[0, 0] = exp[2, 3] = 1
    assert (s.mask() == exp).all()
    bs = s.block_sums()
    assert bs[0, 0] == 5 * 256 and bs[1, 1] == 4 * 256 and bs[2, 3] == 6 * 256
    assert bs.sum() == 15 * 256


def test_intensity_difference_on_coarsest_layer():
    """mask_layer = -1 reads the coarsest octave; one pixel change there is
    enough when its bin holds few layer pixels."""
    W, H = 64, 64
    f0 = np.full((H, W), 90, np.uint8)
    f1 = f0.copy()
    f1[0:8, 0:8] = 190  # c3 pixel (0, 0) moves by 100
    s = oracle.Stream(W, H, N_r=2, N_c=2, O=4, intra=0, T_I=10, t=20,
                      mask_mode=oracle.MASK_ID, mask_layer=-1)
    s.push(f0)
    s.push(f1)
    # c3 is 8x8, bin (0,0) holds 16 of its pixels: mean 100/16 = 6.25 <= 10
    assert (s.mask() == 0).all()
    f2 = f0.copy()
    f2[0:32, 0:32] = 200  # the whole bin: mean 110 > 10
    s.push(f2)
    assert s.mask().tolist() == [[1, 0], [0, 0]]


def test_keypoint_binning_mask_counts_previous_keypoints():
    """Eqs. 3-4: bin active iff it held >= T_H keypoints of D_{n-1}."""
    W, H = 80, 40
    f0 = np.full((H, W), 50, np.uint8)
    # isolated bright pixels: bin (0,0) gets 2, bin (0,1) gets 1, bin (1,3) 3
    pts = [(5, 5), (12, 9), (25, 6), (70, 25), (75, 33), (64, 30)]
    for x, y in pts:
        f0[y, x] = 200
    s = oracle.Stream(W, H, N_r=2, N_c=4, O=1, T_H=2, t=20, mask_mode=oracle.MASK_KB)
    s.push(f0)
    assert len(s.keypoints()) == len(pts)
    s.push(f0)
    exp = np.zeros((2, 4), np.uint8)
    exp[0, 0] = 1
    exp[1, 3] = 1
    assert (s.mask() == exp).all()
    assert s.block_sums().tolist() == [[2, 1, 0, 0], [0, 0, 0, 3]]
    # propagated keypoints of the inactive bin keep their position and score
    kp = s.keypoints()
    prop = kp[kp["flags"] == 1]
    assert [(int(k["x"]), int(k["y"])) for k in prop] == [(25, 6)]


# --------------------------------------------------------------------------
# Eq. 1: propagation


def _stream_pair(**kw):
    return oracle.Stream(**kw), oracle.Stream(**kw)


def test_all_ones_mask_equals_full_detection():
    from paper_1503_06959_gb300 import synth
    src = synth.VideoSource(96, 96, seed=3, n_movers=2, mover_size=20, speed=(2, 3))
    frames = src.frames(4)
    kw = dict(W=96, H=96, N_r=4, N_c=4, O=2, intra=1, T_I=4, t=20)
    a = oracle.Stream(mask_mode=oracle.MASK_ID, **kw)
    b = oracle.Stream(mask_mode=oracle.MASK_FULL, **kw)
    ones = np.ones((4, 4), np.uint8)
    for f in frames:
        a.push(f, mask_override=ones)
        b.push(f)
        assert kp_tuples(a.keypoints()) == kp_tuples(b.keypoints())
        assert (a.keypoints()["flags"] == 0).all()


def test_all_zeros_mask_propagates_everything():
    from paper_1503_06959_gb300 import synth
    src = synth.VideoSource(96, 72, seed=4, n_movers=2, mover_size=20, speed=(3, 3))
    f0, f1 = src.frames(2)
    s = oracle.Stream(96, 72, N_r=3, N_c=4, O=2, intra=1, T_I=4, t=15, mask_mode=oracle.MASK_ID)
    s.push(f0)
    prev = s.keypoints()
    assert len(prev) > 0
    s.push(f1, mask_override=np.zeros((3, 4), np.uint8))
    cur = s.keypoints()
    assert [t[:4] for t in kp_tuples(cur)] == [t[:4] for t in kp_tuples(prev)]
    assert (cur["flags"] == 1).all()


def test_identical_frames_keep_previous_keypoints():
    from paper_1503_06959_gb300 import synth
    f0 = synth.VideoSource(64, 64, seed=9, n_movers=1, mover_size=16).frame(0)
    s = oracle.Stream(64, 64, N_r=4, N_c=4, O=1, T_I=0, t=15, mask_mode=oracle.MASK_ID)
    s.push(f0)
    first = kp_tuples(s.keypoints())
    s.push(f0)  # |d| = 0 everywhere, and 0 > T_I * n fails even for T_I = 0
    assert (s.mask() == 0).all()
    assert [k[:4] for k in kp_tuples(s.keypoints())] == [k[:4] for k in first]


def test_single_active_block_mixes_new_and_old():
    """D_n = (full detections of frame n inside the active bin) united with
    (D_{n-1} outside it); the detections inside use neighbour scores from the
    inactive bins, exactly as the unmasked detector does."""
    from paper_1503_06959_gb300 import synth
    src = synth.VideoSource(96, 96, seed=21, n_movers=3, mover_size=24, speed=(3, 4))
    f0, f1 = src.frames(2)
    kw = dict(W=96, H=96, N_r=3, N_c=3, O=2, intra=1, T_I=4, t=12)
    s = oracle.Stream(mask_mode=oracle.MASK_ID, **kw)
    full = oracle.Stream(mask_mode=oracle.MASK_FULL, **kw)
    s.push(f0)
    full.push(f0)
    d0 = kp_tuples(s.keypoints())
    mask = np.zeros((3, 3), np.uint8)
    mask[1, 1] = 1
    s.push(f1, mask_override=mask)
    full.push(f1)
    scales = [oracle.layer_geom(96, 96, 2, 1, l)[2] for l in range(4)]
    def blk(k):
        return oracle.block_of(k[2], k[1], scales[k[0]], 96, 96, 3, 3)
    exp = [k[:4] + (0,) for k in kp_tuples(full.keypoints()) if blk(k) == 4]
    exp += [k[:4] + (1,) for k in d0 if blk(k) != 4]
    assert kp_tuples(s.keypoints()) == sorted(exp)
    assert any(k[4] == 0 for k in exp) and any(k[4] == 1 for k in exp)


# --------------------------------------------------------------------------
# scale-space non-maximum suppression (Sec. 2, "3x3 scale-space neighbourhood")


def centre_pixel(x, S, S2):
    """The pixel of a layer with scale code S2 whose image footprint
    [x2*S2/2, (x2+1)*S2/2) holds the centre (x + 1/2)*S/2 of pixel x of a
    layer with scale code S, found by search (not by formula)."""
    c = Fraction(2 * x + 1, 2) * Fraction(S, 2)
    x2 = 0
    while Fraction((x2 + 1) * S2, 2) <= c:
        x2 += 1
    assert Fraction(x2 * S2, 2) <= c < Fraction((x2 + 1) * S2, 2)
    return x2


def brute_scale_detect(layers, Ss, t):
    """In-layer strict 3x3 maxima that are also strictly above every score of
    the 3x3 windows (around the centre pixel) of the layers just below and
    above in scale; scores by brute force."""
    sc = []
    for img in layers:
        h, w = img.shape
        sc.append(np.array([[brute_score(img, x, y) for x in range(w)] for y in range(h)], int)
                  if w and h else np.zeros((h, w), int))
    out = []
    for l, img in enumerate(layers):
        h, w = img.shape
        for y in range(h):
            for x in range(w):
                v = sc[l][y, x]
                if v < t:
                    continue
                nb = [sc[l][y + dy, x + dx] if 0 <= y + dy < h and 0 <= x + dx < w else 0
                      for dy in (-1, 0, 1) for dx in (-1, 0, 1) if (dx, dy) != (0, 0)]
                for m in (l - 1, l + 1):
                    if not 0 <= m < len(layers):
                        continue
                    mh, mw = layers[m].shape
                    cx, cy = centre_pixel(x, Ss[l], Ss[m]), centre_pixel(y, Ss[l], Ss[m])
                    nb += [sc[m][cy + dy, cx + dx] if 0 <= cy + dy < mh and 0 <= cx + dx < mw else 0
                           for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
                if all(v > q for q in nb):
                    out.append((l, y, x, int(v)))
    return out


def test_centre_pixel_search_agrees_with_the_integer_map():
    # the oracle maps x -> floor((2x + 1) * S / (2 S2)); the search above
    # finds the containing pixel from the footprints alone
    for S, S2 in ((2, 3), (3, 2), (3, 4), (4, 3), (2, 4), (4, 2), (8, 12), (12, 8)):
        for x in range(40):
            assert centre_pixel(x, S, S2) == ((2 * x + 1) * S) // (2 * S2)


def test_scale_nms_equals_bruteforce_on_small_pyramids():
    rng = np.random.default_rng(77)
    for trial, (O, intra) in enumerate(((2, 1), (3, 0), (2, 0))):
        W, H = 36 + 6 * trial, 30 + 6 * trial
        # plateaus and corners at two sizes, so that coarse layers have corners too
        big = np.kron(rng.integers(0, 4, (H // 6 + 1, W // 6 + 1)), np.ones((6, 6), int))[:H, :W]
        small = rng.integers(0, 3, (H, W))
        img = np.clip(big * 60 + small * 12, 0, 255).astype(np.uint8)
        t = 8
        s = oracle.Stream(W, H, N_r=1, N_c=1, O=O, intra=intra, t=t, mask_mode=oracle.MASK_FULL,
                          nms_scale=1)
        s.push(img)
        got = [(int(k["layer"]), int(k["y"]), int(k["x"]), int(k["score"])) for k in s.keypoints()]
        layers = oracle.pyramid(img, O, intra)
        Ss = [oracle.layer_geom(W, H, O, intra, l)[2] for l in range(len(layers))]
        exp = sorted(brute_scale_detect(layers, Ss, t))
        assert got == exp
        assert len({k[0] for k in got}) > 1, "keypoints on more than one layer"


def test_scale_nms_single_layer_is_in_layer_nms():
    rng = np.random.default_rng(5)
    img = np.clip(rng.normal(128, 60, (40, 52)), 0, 255).astype(np.uint8)
    kps = []
    for ns in (0, 1):
        s = oracle.Stream(52, 40, N_r=2, N_c=2, O=1, intra=0, t=15, mask_mode=oracle.MASK_FULL,
                          nms_scale=ns)
        s.push(img)
        kps.append(kp_tuples(s.keypoints()))
    assert kps[0] == kps[1] and len(kps[0]) > 0


def test_scale_nms_keeps_a_subset_and_removes_only_dominated_points():
    rng = np.random.default_rng(9)
    W, H, O, intra = 96, 72, 3, 1
    img = np.clip(np.round(rng.integers(0, 256, (H, W)) / 32) * 32, 0, 255).astype(np.uint8)
    res = {}
    for ns in (0, 1):
        s = oracle.Stream(W, H, N_r=3, N_c=4, O=O, intra=intra, t=10, mask_mode=oracle.MASK_FULL,
                          nms_scale=ns)
        s.push(img)
        res[ns] = {(int(k["layer"]), int(k["y"]), int(k["x"])): int(k["score"]) for k in s.keypoints()}
    assert set(res[1]) <= set(res[0]) and len(res[1]) < len(res[0])
    layers = oracle.pyramid(img, O, intra)
    Ss = [oracle.layer_geom(W, H, O, intra, l)[2] for l in range(len(layers))]
    for (l, y, x), v in res[0].items():
        if (l, y, x) in res[1]:
            continue
        # removed: some score in an adjacent layer's window is >= v
        found = False
        for m in (l - 1, l + 1):
            if not 0 <= m < len(layers):
                continue
            mh, mw = layers[m].shape
            cx, cy = centre_pixel(x, Ss[l], Ss[m]), centre_pixel(y, Ss[l], Ss[m])
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    if 0 <= cy + dy < mh and 0 <= cx + dx < mw and brute_score(layers[m], cx + dx, cy + dy) >= v:
                        found = True
        assert found, (l, y, x, v)


# --------------------------------------------------------------------------
# Eq. 2 per pixel of every layer (mask mode IDP, option (i) of Sec. 3.1)


def test_pixel_mask_is_eq2_on_every_layer():
    rng = np.random.default_rng(21)
    W, H, O, intra, T_I = 72, 54, 3, 1, 6
    f0 = np.clip(rng.normal(120, 40, (H, W)), 0, 255).astype(np.uint8)
    f1 = f0.copy()
    f1[10:40, 20:60] = np.clip(f1[10:40, 20:60].astype(int) + rng.integers(-30, 31, (30, 40)), 0, 255)
    s = oracle.Stream(W, H, N_r=2, N_c=3, O=O, intra=intra, t=10, T_I=T_I, mask_mode=oracle.MASK_IDP)
    s.push(f0)
    for l in range(oracle.num_layers(O, intra)):
        assert s.pixel_mask(l).all(), "first frame: every pixel active"
    s.push(f1)
    L0, L1 = oracle.pyramid(f0, O, intra), oracle.pyramid(f1, O, intra)
    for l, (a, b) in enumerate(zip(L0, L1)):
        exp = (np.abs(b.astype(int) - a.astype(int)) > T_I).astype(np.uint8)
        np.testing.assert_array_equal(s.pixel_mask(l), exp, err_msg=f"layer {l}")
    assert 0 < s.pixel_mask(0).mean() < 1


def test_pixel_mask_nothing_changes_keeps_everything():
    rng = np.random.default_rng(22)
    f = np.clip(rng.normal(120, 50, (40, 48)), 0, 255).astype(np.uint8)
    s = oracle.Stream(48, 40, N_r=2, N_c=2, O=2, intra=1, t=12, T_I=0, mask_mode=oracle.MASK_IDP)
    s.push(f)
    first = kp_tuples(s.keypoints())
    assert first
    for _ in range(2):
        s.push(f)
        got = kp_tuples(s.keypoints())
        assert [g[:4] for g in got] == [k[:4] for k in first]
        assert all(g[4] == 1 for g in got), "all carried over"


def test_pixel_mask_everything_changes_redetects_everything():
    # +1 on every pixel of c_0 (values <= 200) moves every pyramid pixel by
    # exactly 1: the 2x2 sum grows by 4 and the 3x3 -> 2x2 sum by 9
    rng = np.random.default_rng(23)
    f0 = rng.integers(0, 200, (42, 54)).astype(np.uint8)
    f1 = (f0 + 1).astype(np.uint8)
    kw = dict(N_r=2, N_c=2, O=2, intra=1, t=10)
    s = oracle.Stream(54, 42, T_I=0, mask_mode=oracle.MASK_IDP, **kw)
    s.push(f0)
    s.push(f1)
    full = oracle.Stream(54, 42, mask_mode=oracle.MASK_FULL, **kw)
    full.push(f1)
    assert kp_tuples(s.keypoints()) == kp_tuples(full.keypoints())
    for l in range(4):
        assert s.pixel_mask(l).all()


def test_pixel_mask_detection_equals_bruteforce():
    rng = np.random.default_rng(24)
    W, H, O, intra, T_I, t = 30, 27, 2, 1, 20, 8
    big = np.kron(rng.integers(0, 4, (6, 6)), np.ones((6, 6), int))[:H, :W]
    frames = []
    for n in range(3):
        img = big * 60 + rng.integers(0, 3, (H, W)) * 10
        img[5 + 3 * n:12 + 3 * n, 4:14] = 220 - 30 * n  # a moving plateau
        frames.append(np.clip(img, 0, 255).astype(np.uint8))
    s = oracle.Stream(W, H, N_r=1, N_c=1, O=O, intra=intra, t=t, T_I=T_I, mask_mode=oracle.MASK_IDP)
    prev_layers, prev_kp = None, []
    for f in frames:
        s.push(f)
        layers = oracle.pyramid(f, O, intra)
        if prev_layers is None:
            act = [np.ones(L.shape, bool) for L in layers]
        else:
            act = [np.abs(L.astype(int) - P.astype(int)) > T_I for L, P in zip(layers, prev_layers)]
        exp = [(l, y, x, v, 1) for (l, y, x, v, _) in prev_kp if not act[l][y, x]]
        for l, img in enumerate(layers):
            for (x, y, v) in brute_detect(img, t):
                if act[l][y, x]:
                    exp.append((l, y, x, v, 0))
        exp.sort()
        got = kp_tuples(s.keypoints())
        assert got == exp
        prev_layers, prev_kp = layers, exp
    assert any(k[4] == 1 for k in exp) and any(k[4] == 0 for k in exp)


# --------------------------------------------------------------------------
# masked description (Sec. 2: bits from intensity comparisons of sampled
# pixel pairs; Sec. 3: only detected keypoints are described, carried ones
# keep their descriptors)


def box_sums_padded(img, pad):
    """5x5 sums around every pixel of the replicate-padded image, computed by
    scipy's correlation (an independent routine), exact in int64."""
    ndimage = pytest.importorskip("scipy.ndimage")
    p = np.pad(img.astype(np.int64), pad, mode="edge")
    return ndimage.correlate(p, np.ones((5, 5), np.int64), mode="constant", cval=0)


def library_descriptor(img, x, y, pattern):
    pad = 16
    box = box_sums_padded(img, pad)
    bits = np.zeros(len(pattern), np.uint8)
    for i, (ax, ay, bx, by) in enumerate(pattern.astype(int)):
        bits[i] = box[y + ay + pad, x + ax + pad] < box[y + by + pad, x + bx + pad]
    return np.packbits(bits, bitorder="little")


def test_descriptor_matches_library_box_filter_everywhere():
    rng = np.random.default_rng(11)
    from paper_1503_06959_gb300 import synth
    pattern = np.concatenate([synth.descriptor_pattern(32, seed=5),
                              rng.integers(-13, 14, (32, 4)).astype(np.int8)])
    for h, w in ((29, 37), (7, 5), (40, 33)):
        img = rng.integers(0, 256, (h, w), dtype=np.uint8)
        pts = [(0, 0), (w - 1, h - 1), (w - 1, 0), (0, h - 1), (w // 2, h // 2)]
        pts += [(int(rng.integers(0, w)), int(rng.integers(0, h))) for _ in range(10)]
        for x, y in pts:
            np.testing.assert_array_equal(oracle.describe(img, x, y, pattern),
                                          library_descriptor(img, x, y, pattern), err_msg=f"{w}x{h} at {x},{y}")


def test_descriptor_step_edge_hand_computed():
    img = np.full((40, 40), 10, np.uint8)
    img[:, 20:] = 200
    pattern = np.array([[-6, 0, 6, 0],    # dark left vs bright right: 1
                        [6, 0, -6, 0],    # reversed: 0
                        [0, -6, 0, 6],    # same column, equal sums: 0 (strict)
                        [-1, 0, 0, 0],    # 3 dark + 2 bright columns vs 2 dark + 3 bright: 1
                        [0, 0, -1, 0],    # reversed: 0
                        [3, 3, 3, 3],     # a pair with itself: 0
                        [-13, 13, 13, -13],  # far left vs far right: 1
                        [2, 0, 3, 0]],    # both boxes wholly bright: 0
                       np.int8)
    assert oracle.describe(img, 20, 20, pattern).tolist() == [0b01001001]


def test_descriptor_constant_image_is_all_zeros():
    from paper_1503_06959_gb300 import synth
    img = np.full((30, 30), 77, np.uint8)
    assert not oracle.describe(img, 3, 25, synth.descriptor_pattern(256)).any()


def test_descriptor_rotation_by_90_degrees():
    """Rotating the image, the point and every offset by 90 degrees leaves
    every bit unchanged (the 5x5 boxes and the clamping to the image
    rectangle are symmetric); a swapped or sign-flipped coordinate fails."""
    rng = np.random.default_rng(12)
    img = rng.integers(0, 256, (31, 45), dtype=np.uint8)
    pattern = rng.integers(-13, 14, (64, 4)).astype(np.int8)
    H, W = img.shape
    rot = np.rot90(img)  # rot[r, c] = img[c, W - 1 - r]: (x, y) -> (y, W - 1 - x)
    rpat = np.stack([pattern[:, 1], -pattern[:, 0], pattern[:, 3], -pattern[:, 2]], axis=1).astype(np.int8)
    for x, y in ((0, 0), (44, 30), (10, 3), (22, 15), (40, 28)):
        np.testing.assert_array_equal(oracle.describe(rot, y, W - 1 - x, rpat),
                                      oracle.describe(img, x, y, pattern))


def _describe_all(frame, kp, O, intra, pattern):
    layers = oracle.pyramid(frame, O, intra)
    return np.array([oracle.describe(layers[k["layer"]], int(k["x"]), int(k["y"]), pattern) for k in kp]
                    ).reshape(len(kp), -1)


@pytest.mark.parametrize("mode", ["ID", "IDP", "KB"])
def test_masked_description_describes_new_and_carries_old(mode):
    from paper_1503_06959_gb300 import synth
    src = synth.VideoSource(96, 96, seed=23, n_movers=3, mover_size=24, speed=(3, 4))
    frames = src.frames(4)
    pattern = synth.descriptor_pattern(128, seed=3)
    kw = dict(N_r=3, N_c=3, O=2, intra=1, T_I=4, t=12, pattern=pattern)
    modes = {"ID": oracle.MASK_ID, "IDP": oracle.MASK_IDP, "KB": oracle.MASK_KB}
    s = oracle.Stream(96, 96, mask_mode=modes[mode], T_H=2, **kw)
    one = np.zeros((3, 3), np.uint8)
    one[1, 1] = 1
    prev_kp, prev_d = None, None
    seen_carried_changed = False
    for n, f in enumerate(frames):
        s.push(f, mask_override=one if (mode == "ID" and n > 0) else None)
        kp, d = s.keypoints(), s.descriptors()
        assert d.shape == (len(kp), 16)
        here = _describe_all(f, kp, 2, 1, pattern)
        new = kp["flags"] == 0
        np.testing.assert_array_equal(d[new], here[new])
        if n == 0:
            assert new.all()
        else:
            if mode != "KB":
                assert (~new).any() and new.any()
            index = {(int(k["layer"]), int(k["y"]), int(k["x"])): i for i, k in enumerate(prev_kp)}
            for i in np.flatnonzero(~new):
                k = kp[i]
                j = index[(int(k["layer"]), int(k["y"]), int(k["x"]))]
                np.testing.assert_array_equal(d[i], prev_d[j])
                seen_carried_changed |= not np.array_equal(d[i], here[i])
        prev_kp, prev_d = kp, d
    # the carried descriptors come from the frame that detected them, not
    # from the current pixels (which moved under some of them; keypoint
    # binning carries only sparse, mostly static bins)
    assert seen_carried_changed or mode == "KB"


def test_description_is_set_before_the_first_frame_only():
    from paper_1503_06959_gb300 import synth
    s = oracle.Stream(64, 48, N_r=2, N_c=2, O=1, t=15)
    s.push(synth.VideoSource(64, 48, seed=1).frame(0))
    lib = oracle._load()
    pat = synth.descriptor_pattern(64)
    assert lib.orc_stream_set_descriptor(s._h, oracle._ptr(pat), 64) == -1
    with pytest.raises(ValueError):
        s.descriptors()
