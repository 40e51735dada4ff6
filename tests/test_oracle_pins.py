"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test pins part of the definition in Sec. 2 of the paper (Alg. 1, Eqs. 4-5):
hand-worked cases, the pair-count invariant, permutation and translation
invariance, the ideal-gas closed form, a brute-force image search for
triclinic boxes and an exact rational recomputation of r^2 and of the bin on
tiny inputs.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import workloads as w

NONE, ORTHO, TRIC = w.BOX_NONE, w.BOX_ORTHO, w.BOX_TRICLINIC


def hist(oracle_mod, coords, offsets, box_type, box, r_max, nbins):
    return oracle_mod.histogram(np.asarray(coords, dtype=np.float32), np.asarray(offsets), box_type,
                                box, r_max, nbins, nthreads=4)


# ---------------------------------------------------------------- hand-worked cases


def test_hand_single_pair_bin(oracle_mod):
    # r = 1.5, dr = 1 -> bin 1 (Eq. 4: r_k <= r < r_k + dr)
    h = hist(oracle_mod, [[0, 0, 0], [1.5, 0, 0]], [0, 2], NONE, None, 4.0, 4)
    assert h.tolist() == [[0, 1, 0, 0]]


def test_hand_edge_goes_to_upper_bin(oracle_mod):
    # 3-4-5 triangle: r = 5 exactly on the edge between bins 4 and 5 -> bin 5 (half-open bins)
    h = hist(oracle_mod, [[0, 0, 0], [3, 4, 0]], [0, 2], NONE, None, 10.0, 10)
    assert h[0].tolist() == [0, 0, 0, 0, 0, 1, 0, 0, 0, 0]


def test_hand_r_equal_rmax_dropped(oracle_mod):
    h = hist(oracle_mod, [[0, 0, 0], [3, 4, 0]], [0, 2], NONE, None, 5.0, 5)
    assert h.sum() == 0
    h = hist(oracle_mod, [[0, 0, 0], [3, 4, 0]], [0, 2], NONE, None, 5.0000001, 5)
    assert h[0].tolist() == [0, 0, 0, 0, 1]


def test_hand_ortho_minimum_image(oracle_mod):
    box = w.ortho_box(10.0)
    # 1 and 9 on a ring of 10 are 2 apart
    h = hist(oracle_mod, [[1, 0, 0], [9, 0, 0]], [0, 2], ORTHO, box, 5.0, 5)
    assert h[0].tolist() == [0, 0, 1, 0, 0]
    # half-box separation: r = 5 either way
    assert oracle_mod.pair_r2([0, 0, 0], [5, 0, 0], ORTHO, box) == 25.0
    # 15 and 25 apart: nint rounds half to even (1.5 -> 2, 2.5 -> 2) -> |d'| = 5
    assert oracle_mod.pair_r2([0, 0, 0], [15, 0, 0], ORTHO, box) == 25.0
    assert oracle_mod.pair_r2([0, 0, 0], [25, 0, 0], ORTHO, box) == 25.0
    # two axes wrapped: d = (9, 9.5, 0) -> (-1, -0.5, 0)
    assert oracle_mod.pair_r2([0.5, 0, 0], [9.5, 9.5, 0], ORTHO, box) == 1.25
    # coordinates outside the primary cell are wrapped by Eq. 5 as well
    assert oracle_mod.pair_r2([-31, 0, 0], [2, 0, 0], ORTHO, box) == 9.0
    # each axis uses its own length
    box3 = w.ortho_box(10.0, 20.0, 40.0)
    assert oracle_mod.pair_r2([0, 0, 0], [9, 19, 39], ORTHO, box3) == 3.0


def test_hand_triclinic_lattice_vector(oracle_mod):
    box = np.array([8.0, 2.0, -1.5, 0.0, 8.0, 2.5, 0.0, 0.0, 8.0])
    p = np.array([1.0, 2.0, 3.0])
    a, b, c = box.reshape(3, 3).T
    # a point one lattice vector a+b away is the same point: r = 0
    assert oracle_mod.pair_r2(p, p + a + b, TRIC, box) == 0.0
    assert oracle_mod.pair_r2(p, p - a + 2 * b - c, TRIC, box) == 0.0
    # a lattice vector plus a small offset: r = |offset|
    assert oracle_mod.pair_r2(p, p + a + b + np.array([0.25, 0, 0]), TRIC, box) == 0.0625
    assert oracle_mod.pair_r2(p, p + c + np.array([0.0, 0.5, 0.0]), TRIC, box) == 0.25


def test_hand_two_species_order(oracle_mod):
    # A = {(0,0,0)}, B = {(1,0,0), (2,0,0)}: AA has no pair, AB has r=1 and r=2, BB has r=1
    h = hist(oracle_mod, [[0, 0, 0], [1, 0, 0], [2, 0, 0]], [0, 1, 3], NONE, None, 4.0, 4)
    assert h.tolist() == [[0, 0, 0, 0], [0, 1, 1, 0], [0, 1, 0, 0]]


def test_hand_three_species_histogram_order(oracle_mod):
    # species placed so that every species pair has its own distance:
    # AA=1, AB=10, AC=20(ish), BB=2, BC=..., CC=3 -> order (0,0),(0,1),(0,2),(1,1),(1,2),(2,2)
    A = [[0, 0, 0], [1, 0, 0]]
    B = [[0, 10, 0], [2, 10, 0]]
    C = [[0, 0, 30], [3, 0, 30]]
    x = A + B + C
    h = hist(oracle_mod, x, [0, 2, 4, 6], NONE, None, 64.0, 64)
    nz = [sorted(np.repeat(np.arange(64), h[k].astype(np.int64)).tolist()) for k in range(6)]
    d = lambda p, q: int(math.floor(math.dist(p, q)))
    expect = [
        [d(A[0], A[1])],
        sorted(d(p, q) for p in A for q in B),
        sorted(d(p, q) for p in A for q in C),
        [d(B[0], B[1])],
        sorted(d(p, q) for p in B for q in C),
        [d(C[0], C[1])],
    ]
    assert nz == expect


def test_hand_single_species_pair_histogram(oracle_mod):
    # histogram_one(a, c) is the (a, c) histogram alone: the hand-worked
    # three-species frame above, and the two-species frame's AB pair
    A = [[0, 0, 0], [1, 0, 0]]
    B = [[0, 10, 0], [2, 10, 0]]
    C = [[0, 0, 30], [3, 0, 30]]
    x = np.array(A + B + C, dtype=np.float32)
    d = lambda p, q: int(math.floor(math.dist(p, q)))
    want = {(0, 1): [d(p, q) for p in A for q in B], (1, 2): [d(p, q) for p in B for q in C],
            (2, 2): [d(C[0], C[1])]}
    for (a, c), ds in want.items():
        h = oracle_mod.histogram_one(x, [0, 2, 4, 6], NONE, None, 64.0, 64, a, c)
        assert sorted(np.repeat(np.arange(64), h.astype(np.int64)).tolist()) == sorted(ds)
    h = oracle_mod.histogram_one(np.array([[0, 0, 0], [1, 0, 0], [2, 0, 0]], np.float32), [0, 1, 3], NONE, None,
                                 4.0, 4, 0, 1)
    assert h.tolist() == [0, 1, 1, 0]
    with pytest.raises(ValueError):
        oracle_mod.histogram_one(x, [0, 2, 4, 6], NONE, None, 64.0, 64, 1, 0)


@pytest.mark.parametrize("box_type", [NONE, ORTHO, TRIC])
def test_single_species_pair_matches_all_pairs(oracle_mod, box_type):
    # each species-pair histogram alone equals its row of the full set
    box = {NONE: None, ORTHO: w.ortho_box(9.0, 8.0, 10.0), TRIC: w.triclinic_box(9, 9, 9, *w.C3_ANGLES)}[box_type]
    f = w.uniform_frame(71, 900, box_type, box if box is not None else w.ortho_box(9.0), 4.0, 200, n_species=3)
    full = oracle_mod.histogram_frame(f)
    k = 0
    for a in range(3):
        for c in range(a, 3):
            one = oracle_mod.histogram_one(f.coords, f.offsets, f.box_type, f.box, f.r_max, f.nbins, a, c)
            assert np.array_equal(one, full[k]), (a, c)
            k += 1


def test_empty_species_and_tiny_frames(oracle_mod):
    h = hist(oracle_mod, [[0, 0, 0], [1, 0, 0]], [0, 0, 2, 2], NONE, None, 4.0, 4)
    assert h.shape == (6, 4)
    assert h.sum() == 1 and h[3, 1] == 1  # only (1,1) has a pair
    h = hist(oracle_mod, np.zeros((0, 3)), [0, 0], NONE, None, 1.0, 3)
    assert h.tolist() == [[0, 0, 0]]
    h = hist(oracle_mod, [[0, 0, 0]], [0, 1], NONE, None, 1.0, 1)
    assert h.tolist() == [[0]]


def test_invalid_arguments_rejected(oracle_mod):
    with pytest.raises(ValueError):
        hist(oracle_mod, [[0, 0, 0], [1, 0, 0]], [0, 1], NONE, None, 1.0, 4)  # offsets end != n
    with pytest.raises(ValueError):
        hist(oracle_mod, [[0, 0, 0], [1, 0, 0]], [0, 2], NONE, None, 0.0, 4)
    with pytest.raises(ValueError):
        hist(oracle_mod, [[0, 0, 0], [1, 0, 0]], [0, 2], NONE, None, 1.0, 0)


# ---------------------------------------------------------------- invariants


def test_pair_count_invariant_nobox_config(oracle_mod):
    f = w.config_small_nobox(seed=3)
    h = oracle_mod.histogram_frame(f, nthreads=4)
    assert int(h.sum()) == 2000 * 1999 // 2 == 1_999_000


def test_pair_count_invariant_all_in_range_periodic(oracle_mod):
    # the longest minimum-image vector in a cube of side L is L*sqrt(3)/2
    f = w.uniform_frame(5, 700, ORTHO, w.ortho_box(10.0), 10.0 * math.sqrt(3) / 2 + 1e-3, 97,
                        n_species=2)
    h = oracle_mod.histogram_frame(f, nthreads=4)
    na, nb = f.species_sizes()
    assert h[0].sum() == na * (na - 1) // 2
    assert h[1].sum() == na * nb
    assert h[2].sum() == nb * (nb - 1) // 2


def test_pair_count_matches_brute_count_in_range(oracle_mod):
    f = w.uniform_frame(6, 400, ORTHO, w.ortho_box(12.0, 9.0, 15.0), 4.0, 40)
    h = oracle_mod.histogram_frame(f, nthreads=4)
    x = f.coords.astype(np.float64)
    d = x[None, :, :] - x[:, None, :]
    L = np.array([12.0, 9.0, 15.0])
    d -= L * np.round(d / L)
    r = np.sqrt((d ** 2).sum(-1))
    iu = np.triu_indices(f.n, 1)
    assert int(h.sum()) == int((r[iu] < 4.0).sum())


@pytest.mark.parametrize("box_type", [NONE, ORTHO, TRIC])
def test_permutation_invariance_bit_exact(oracle_mod, box_type):
    if box_type == TRIC:
        box = w.triclinic_box(20, 20, 20, *w.C3_ANGLES)
        r_max = 0.95 * w.box_heights(box).min() / 2
    elif box_type == ORTHO:
        box, r_max = w.ortho_box(20.0), 10.0
    else:
        box, r_max = np.zeros(9), 30.0
    f = w.uniform_frame(11, 600, box_type, box if box_type else w.ortho_box(20.0), r_max, 300,
                        n_species=2)
    h0 = oracle_mod.histogram_frame(f, nthreads=4)
    rng = np.random.default_rng(0)
    x = f.coords.copy()
    na = f.species_sizes()[0]
    x[:na] = x[rng.permutation(na)]
    x[na:] = x[na + rng.permutation(f.n - na)]
    h1 = hist(oracle_mod, x, f.offsets, box_type, f.box, r_max, 300)
    assert np.array_equal(h0, h1)
    # swapping the two species swaps AA and BB and leaves AB unchanged (d -> -d exactly)
    xs = np.concatenate([x[na:], x[:na]])
    h2 = hist(oracle_mod, xs, [0, f.n - na, f.n], box_type, f.box, r_max, 300)
    assert np.array_equal(h2[0], h1[2]) and np.array_equal(h2[2], h1[0])
    assert np.array_equal(h2[1], h1[1])


def _dyadic(rng, n, scale):
    # multiples of 2^-10 with |x| < 2^13: every difference and every shift below is exact
    return (np.round(rng.random((n, 3)) * scale * 1024) / 1024).astype(np.float32)


def test_translation_invariance_nobox_bit_exact(oracle_mod):
    rng = np.random.default_rng(1)
    x = _dyadic(rng, 500, 20.0)
    h0 = hist(oracle_mod, x, [0, 500], NONE, None, 25.0, 250)
    shift = np.array([1037.125, -517.5, 3.0009765625], dtype=np.float32)
    h1 = hist(oracle_mod, x + shift, [0, 500], NONE, None, 25.0, 250)
    assert np.array_equal(h0, h1) and h0.sum() > 0


def test_translation_by_box_vector_bit_exact(oracle_mod):
    rng = np.random.default_rng(2)
    box = w.ortho_box(64.0)
    x = _dyadic(rng, 500, 64.0)
    h0 = hist(oracle_mod, x, [0, 250, 500], ORTHO, box, 32.0, 320)
    x1 = x.copy()
    x1[::3] += np.float32(64.0)  # move a third of the particles by one box vector
    x1[1::3, 1] -= np.float32(128.0)
    h1 = hist(oracle_mod, x1, [0, 250, 500], ORTHO, box, 32.0, 320)
    assert np.array_equal(h0, h1)
    # dyadic triclinic cell (reduced: |bx|,|cx| <= ax/2, |cy| <= by/2)
    tbox = np.array([32.0, 8.0, -6.0, 0.0, 32.0, 10.0, 0.0, 0.0, 32.0])
    a, b, c = tbox.reshape(3, 3).T
    x = _dyadic(rng, 400, 30.0)
    h0 = hist(oracle_mod, x, [0, 400], TRIC, tbox, 14.0, 140)
    x1 = x.copy()
    x1[::2] += (a - 2 * b + c).astype(np.float32)
    h1 = hist(oracle_mod, x1, [0, 400], TRIC, tbox, 14.0, 140)
    assert np.array_equal(h0, h1) and h0.sum() > 0


def test_ortho_box_as_triclinic_equals_ortho_path(oracle_mod):
    # with a power-of-two side 1/L is exact, so both forms of Eq. 5 do the same arithmetic
    box = w.ortho_box(32.0)
    f = w.uniform_frame(7, 800, ORTHO, box, 16.0, 160, n_species=2)
    h_o = oracle_mod.histogram_frame(f, nthreads=4)
    h_t = hist(oracle_mod, f.coords, f.offsets, TRIC, box, 16.0, 160)
    assert np.array_equal(h_o, h_t)


# ---------------------------------------------------------------- closed form


def _ideal_gas_chi2(h, n_pairs, r_max, nbins, volume):
    dr = r_max / nbins
    edges = np.arange(nbins + 1) * dr
    expect = n_pairs * (4.0 * math.pi / 3.0) * (edges[1:] ** 3 - edges[:-1] ** 3) / volume
    return float((((h - expect) ** 2) / expect).sum()), expect


@pytest.mark.parametrize("box_type", [ORTHO, TRIC])
def test_ideal_gas_closed_form(oracle_mod, box_type):
    # uniform particles, r_max <= h_min/2: E[count_k] = P (4 pi / 3)(r_{k+1}^3 - r_k^3) / V
    if box_type == ORTHO:
        box = w.ortho_box(30.0, 24.0, 36.0)
    else:
        box = w.triclinic_box(30.0, 30.0, 30.0, *w.C3_ANGLES)
    r_max = 0.95 * w.box_heights(box).min() / 2
    nbins = 40
    f = w.uniform_frame(21, 4000, box_type, box, r_max, nbins)
    h = oracle_mod.histogram_frame(f, nthreads=8)[0].astype(np.float64)
    chi2, expect = _ideal_gas_chi2(h, f.n_pairs(), r_max, nbins, w.box_volume(box))
    # counts are close to Poisson; chi^2 with 40 dof has its 1e-6 upper tail near 100
    assert chi2 < 100.0, chi2
    assert abs(h.sum() / expect.sum() - 1.0) < 0.01


def test_ideal_gas_detects_missing_minimum_image(oracle_mod):
    # control: the same statistic rejects the non-periodic count of the same particles
    box = w.ortho_box(30.0)
    f = w.uniform_frame(21, 4000, ORTHO, box, 14.0, 40)
    h = hist(oracle_mod, f.coords, f.offsets, NONE, None, 14.0, 40)[0].astype(np.float64)
    chi2, _ = _ideal_gas_chi2(h, f.n_pairs(), 14.0, 40, w.box_volume(box))
    assert chi2 > 1000.0


# ---------------------------------------------------------------- triclinic brute force


def _brute_min_image_r2(x, box, reach=3):
    """Minimum over lattice shifts m in {-reach..reach}^3 of |xj - xi + B m|^2, no wrapping."""
    m = w.box_matrix(box)
    rng_ = np.arange(-reach, reach + 1)
    shifts = np.stack(np.meshgrid(rng_, rng_, rng_, indexing="ij"), -1).reshape(-1, 3) @ m.T
    x = x.astype(np.float64)
    iu, ju = np.triu_indices(len(x), 1)
    d = x[ju] - x[iu]
    best = np.full(len(iu), np.inf)
    for s in shifts:
        best = np.minimum(best, ((d + s) ** 2).sum(-1))
    return iu, ju, best


@pytest.mark.parametrize("angles", [w.C3_ANGLES, (60.0, 60.0, 90.0), (75.0, 105.0, 95.0)])
def test_triclinic_27_images_equal_brute_force(oracle_mod, angles):
    box = w.triclinic_box(20.0, 22.0, 19.0, *angles)
    rng = np.random.default_rng(4)
    # positions spread over several cells so Eq. 5 has to wrap by more than one box vector
    s = rng.random((300, 3)) * 3.0 - 1.0
    x = (w.box_matrix(box) @ s.T).T.astype(np.float32)
    iu, ju, brute = _brute_min_image_r2(x, box)
    ours = oracle_mod.pairs_r2(x, iu, ju, TRIC, box)
    h_half = w.box_heights(box).min() / 2
    inside = brute < h_half ** 2
    assert inside.sum() > 1000
    # below half the smallest plane spacing the image is unique: same vector up to rounding
    np.testing.assert_allclose(ours[inside], brute[inside], rtol=1e-12, atol=1e-9)
    # everywhere the 27-image minimum is never shorter than the true minimum image
    assert np.all(ours >= brute * (1 - 1e-12) - 1e-9)


# ---------------------------------------------------------------- exact rational recomputation


def _nint_even(q: Fraction) -> int:
    fl = math.floor(q)
    rem = q - fl
    if rem > Fraction(1, 2):
        return fl + 1
    if rem < Fraction(1, 2):
        return fl
    return fl if fl % 2 == 0 else fl + 1


def _exact_r2(xi, xj, box_type, box):
    d = [Fraction(float(xj[c])) - Fraction(float(xi[c])) for c in range(3)]
    if box_type == ORTHO:
        L = [Fraction(float(box[0])), Fraction(float(box[4])), Fraction(float(box[8]))]
        d = [d[c] - L[c] * _nint_even(d[c] / L[c]) for c in range(3)]
        return sum(v * v for v in d)
    if box_type == TRIC:
        B = [[Fraction(float(box[3 * r + c])) for c in range(3)] for r in range(3)]
        sz = d[2] / B[2][2]
        sy = (d[1] - B[1][2] * sz) / B[1][1]
        sx = (d[0] - B[0][1] * sy - B[0][2] * sz) / B[0][0]
        k = [_nint_even(sx), _nint_even(sy), _nint_even(sz)]
        dd = [d[r] - sum(B[r][c] * k[c] for c in range(3)) for r in range(3)]
        best = None
        for mx in (-1, 0, 1):
            for my in (-1, 0, 1):
                for mz in (-1, 0, 1):
                    m = (mx, my, mz)
                    e = [dd[r] + sum(B[r][c] * m[c] for c in range(3)) for r in range(3)]
                    v = sum(t * t for t in e)
                    best = v if best is None or v < best else best
        return best
    return sum(v * v for v in d)


def _exact_bin(r2: Fraction, r_max: float, nbins: int):
    # floor(nbins * sqrt(r2) / r_max) exactly: floor(sqrt(p/q)) = isqrt(p*q) // q
    v = Fraction(nbins) ** 2 * r2 / Fraction(r_max) ** 2
    k = math.isqrt(v.numerator * v.denominator) // v.denominator
    t = math.sqrt(float(v))
    return min(k, nbins), t


@pytest.mark.parametrize("box_type", [NONE, ORTHO, TRIC])
def test_exact_rational_recomputation(oracle_mod, box_type):
    rng = np.random.default_rng(10 + box_type)
    if box_type == ORTHO:
        box = w.ortho_box(7.3, 5.9, 9.1)
        s = rng.random((60, 3)) * 2.0 - 0.5
        x = (s * np.array([7.3, 5.9, 9.1])).astype(np.float32)
        r_max, nbins = 2.9, 1000
    elif box_type == TRIC:
        box = w.triclinic_box(7.0, 8.0, 6.5, 75.0, 105.0, 95.0)
        s = rng.random((60, 3)) * 2.0 - 0.5
        x = (w.box_matrix(box) @ s.T).T.astype(np.float32)
        r_max, nbins = 0.95 * w.box_heights(box).min() / 2, 997
    else:
        box = None
        x = (rng.random((60, 3)) * 5.0 - 2.5).astype(np.float32)
        r_max, nbins = 4.1, 1001
    iu, ju = np.triu_indices(len(x), 1)
    ours_r2 = oracle_mod.pairs_r2(x, iu, ju, box_type, box)
    checked = 0
    for p in range(len(iu)):
        ex = _exact_r2(x[iu[p]], x[ju[p]], box_type, box)
        assert abs(ours_r2[p] - float(ex)) <= 4e-16 * float(ex) + 1e-300
        kb, t = _exact_bin(ex, r_max, nbins)
        if abs(t - round(t)) < 1e-9:
            continue  # FP64 rounding may decide an exact-edge case either way
        assert oracle_mod.bin_of(ours_r2[p], r_max, nbins) == kb
        checked += 1
    assert checked > 1700
    # and the histogram counts exactly those bins
    h = hist(oracle_mod, x, [0, len(x)], box_type, box, r_max, nbins)[0]
    direct = np.zeros(nbins, dtype=np.uint64)
    for v in ours_r2:
        k = oracle_mod.bin_of(v, r_max, nbins)
        if k < nbins:
            direct[k] += 1
    assert np.array_equal(h, direct)


def test_bin_function_monotone_and_half_open(oracle_mod):
    # bin(r^2) never decreases with r^2 and each edge kappa*dr belongs to bin kappa
    r_max, nbins = 3.0, 12
    for k in range(1, nbins):
        edge = k * r_max / nbins
        assert oracle_mod.bin_of(edge * edge, r_max, nbins) in (k - 1, k)
    r2 = np.sort(np.random.default_rng(0).random(5000) * 10.0)
    bins = [oracle_mod.bin_of(v, r_max, nbins) for v in r2]
    assert all(b0 <= b1 for b0, b1 in zip(bins, bins[1:]))
    assert oracle_mod.bin_of(r_max * r_max, r_max, nbins) == nbins


# ---------------------------------------------------------------- g(r) normalisation (Eq. 1)


def test_rdf_hand_shells(oracle_mod):
    # dr = 1: the shells hold (4 pi / 3)(1, 7, 19); at pair density 3 / (4 pi) a uniform
    # distribution puts 1, 7 and 19 pairs in them, so these counts give g = 1 in every bin
    g = oracle_mod.rdf(np.array([[1, 7, 19]], np.uint64), 3.0, [3.0 / (4.0 * math.pi)], 1)
    assert np.allclose(g, 1.0, rtol=1e-14, atol=0)


def test_rdf_frames_and_density_scale(oracle_mod):
    c = np.array([[5, 0, 40, 123], [2, 9, 0, 77]], np.uint64)
    g1 = oracle_mod.rdf(c, 2.0, [0.5, 0.25], 1)
    # counts summed over 4 identical frames, divided by 4 frames: the same g
    assert np.allclose(oracle_mod.rdf(c * np.uint64(4), 2.0, [0.5, 0.25], 4), g1, rtol=1e-14, atol=0)
    # twice the pair density: half the g
    assert np.allclose(oracle_mod.rdf(c, 2.0, [1.0, 0.5], 1), 0.5 * g1, rtol=1e-14, atol=0)
    # bin k of width dr = r_max / nbins holds (4 pi / 3) dr^3 (3k^2 + 3k + 1) of volume
    dr = 0.5
    shell = 4.0 * math.pi / 3.0 * dr ** 3 * np.array([1.0, 7.0, 19.0, 37.0])
    assert np.allclose(g1[0], c[0] / (0.5 * shell), rtol=1e-13, atol=0)


def test_rdf_ideal_gas_is_one(oracle_mod):
    # uniform particles in a periodic box (r_max <= L/2): g = 1 up to counting noise, for the
    # two intra-species histograms (N_a(N_a-1)/2 / V) and the inter-species one (N_a N_b / V)
    box = w.ortho_box(24.0)
    r_max, nbins = 12.0, 30
    f = w.uniform_frame(22, 6000, ORTHO, box, r_max, nbins, n_species=2)
    h = oracle_mod.histogram_frame(f, nthreads=8)
    na, nb = f.species_sizes()
    V = w.box_volume(box)
    dens = [na * (na - 1) / 2 / V, na * nb / V, nb * (nb - 1) / 2 / V]
    g = oracle_mod.rdf(h, r_max, dens, 1)
    dr = r_max / nbins
    k = np.arange(nbins, dtype=np.float64)
    for hh in range(3):
        expect = dens[hh] * 4.0 * math.pi / 3.0 * dr ** 3 * (3 * k * k + 3 * k + 1)
        z = (g[hh] - 1.0) * np.sqrt(expect)  # Poisson: sd of g is 1/sqrt(expected count)
        assert np.all(np.abs(z) < 6.0), np.abs(z).max()
        assert abs((g[hh] * expect).sum() / expect.sum() - 1.0) < 0.01


# ---------------------------------------------------------------- binary64 input coordinates


@pytest.mark.parametrize("box_type", [NONE, ORTHO, TRIC])
def test_f64_input_equals_f32_input_on_float_values(oracle_mod, box_type):
    # binary64 coordinates that hold float32 values: the distance vector is exact in
    # both definitions, so every bin agrees with the (pinned) float32-input oracle
    box = {NONE: None, ORTHO: w.ortho_box(9.0, 7.5, 11.0), TRIC: w.triclinic_box(9.0, 9.0, 9.0, *w.C3_ANGLES)}
    f = w.uniform_frame(70 + box_type, 700, box_type, box[box_type] if box_type != NONE else w.ortho_box(8.0),
                        3.9, 777, n_species=3)
    h32 = oracle_mod.histogram(f.coords, f.offsets, box_type, box[box_type], f.r_max, f.nbins, nthreads=4)
    h64 = oracle_mod.histogram(f.coords.astype(np.float64), f.offsets, box_type, box[box_type], f.r_max, f.nbins,
                               nthreads=4)
    assert np.array_equal(h32, h64)


@pytest.mark.parametrize("box_type", [NONE, ORTHO, TRIC])
def test_f64_input_exact_rational_bins(oracle_mod, box_type):
    # binary64 coordinates with all 53 bits used: the histogram equals the exact
    # rational bins (pairs within 1e-9 of an edge, where rounding may decide either
    # way, are avoided by construction)
    rng = np.random.default_rng(80 + box_type)
    if box_type == ORTHO:
        box = w.ortho_box(7.3, 5.9, 9.1)
        x = (rng.random((70, 3)) * 2.0 - 0.5) * np.array([7.3, 5.9, 9.1])
        r_max, nbins = 2.9, 1000
    elif box_type == TRIC:
        box = w.triclinic_box(7.0, 8.0, 6.5, 75.0, 105.0, 95.0)
        x = (w.box_matrix(box) @ (rng.random((70, 3)) * 2.0 - 0.5).T).T
        r_max, nbins = 0.95 * w.box_heights(box).min() / 2, 997
    else:
        box = None
        x = rng.random((70, 3)) * 5.0 - 2.5
        r_max, nbins = 4.1, 1001
    x = np.ascontiguousarray(x, dtype=np.float64)
    assert np.any(x.astype(np.float32).astype(np.float64) != x)  # not float32 values
    # r^2 itself against the exact rational value: each component of the distance
    # vector now carries rounding errors of the coordinate magnitude X (the
    # subtraction and, with a box, the image steps): |dr^2| <= 2 |d'| e + e^2 per
    # component with e <= 8 * 2^-53 * X, plus a few relative roundings of the sum.
    # Coordinates rounded to float32 (errors 2^-24 X) fail this by far.
    iu, ju = np.triu_indices(len(x), 1)
    ours = oracle_mod.pairs_r2(x, iu, ju, box_type, box)
    X = float(np.abs(x).max()) + (0.0 if box is None else float(np.abs(box).sum()))
    e = 8.0 * 2.0 ** -53 * X
    for p in range(len(iu)):
        ex = float(_exact_r2(x[iu[p]], x[ju[p]], box_type, box))
        tol = 2.0 * math.sqrt(3.0 * ex) * e + 3.0 * e * e + 4e-16 * ex
        assert abs(ours[p] - ex) <= tol, (p, ours[p], ex)
    direct = np.zeros(nbins, dtype=np.uint64)
    for i in range(len(x)):
        for j in range(i + 1, len(x)):
            kb, t = _exact_bin(_exact_r2(x[i], x[j], box_type, box), r_max, nbins)
            assert abs(t - round(t)) > 1e-9 or t > nbins + 1
            if kb < nbins:
                direct[kb] += 1
    h = oracle_mod.histogram(x, [0, len(x)], box_type, box, r_max, nbins, nthreads=4)[0]
    assert np.array_equal(h, direct)


def test_f64_input_dyadic_translation(oracle_mod):
    # multiples of 2^-30 below 2^8: every difference is exact in binary64, so a
    # translation by a dyadic box vector leaves every bin unchanged
    rng = np.random.default_rng(90)
    box = w.ortho_box(64.0, 48.0, 80.0)
    x = np.floor(rng.random((600, 3)) * np.array([64.0, 48.0, 80.0]) * 2.0 ** 30) / 2.0 ** 30
    h0 = oracle_mod.histogram(x, [0, 200, 600], ORTHO, box, 23.0, 900, nthreads=4)
    h1 = oracle_mod.histogram(x + np.array([64.0, -48.0, 160.0]), [0, 200, 600], ORTHO, box, 23.0, 900,
                              nthreads=4)
    assert np.array_equal(h0, h1)
