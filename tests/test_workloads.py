"""The seeded input recipe (the shapes, sizes and distributions of the paper's
workloads that the tests and the bench use) against its written description."""
import math

import numpy as np
import pytest

import workloads as w


def fractional(x, box):
    return np.linalg.solve(w.box_matrix(box), x.astype(np.float64).T).T


def angles_of(box):
    m = w.box_matrix(box)
    a, b, c = m[:, 0], m[:, 1], m[:, 2]
    ang = lambda u, v: math.degrees(math.acos(float(u @ v) / (np.linalg.norm(u) * np.linalg.norm(v))))
    return (np.linalg.norm(a), np.linalg.norm(b), np.linalg.norm(c)), (ang(b, c), ang(a, c), ang(a, b))


def test_c1_small_nobox():
    f = w.config_small_nobox(seed=1)
    assert f.n == 2000 and f.box_type == w.BOX_NONE and f.nbins == 1000 and f.r_max == 17.33
    assert list(f.offsets) == [0, 2000]
    assert f.coords.dtype == np.float32 and f.coords.min() >= 0.0 and f.coords.max() < 10.0
    assert f.r_max > 10.0 * math.sqrt(3.0)  # every pair in range
    assert f.n_pairs() == 1_999_000


def test_c2_ortho_two_species():
    f = w.config_ortho_two_species(seed=1)
    assert f.n == 100_000 and list(f.offsets) == [0, 50_000, 100_000]
    assert f.box_type == w.BOX_ORTHO and np.allclose(w.box_matrix(f.box), np.diag([60.0] * 3))
    assert f.r_max == 30.0 and f.nbins == 10_000
    assert f.coords.min() >= 0.0 and f.coords.max() < 60.0


def test_c3_triclinic_clusters():
    f = w.config_triclinic_clusters(seed=1)
    assert f.n == 500_000 and f.box_type == w.BOX_TRICLINIC and f.r_max == 35.0 and f.nbins == 20_000
    lengths, angs = angles_of(f.box)
    assert np.allclose(lengths, 80.0) and np.allclose(angs, w.C3_ANGLES)
    m = w.box_matrix(f.box)
    assert m[1, 0] == 0 and m[2, 0] == 0 and m[2, 1] == 0  # upper triangular
    assert abs(m[0, 1]) <= m[0, 0] / 2 and abs(m[0, 2]) <= m[0, 0] / 2 and abs(m[1, 2]) <= m[1, 1] / 2
    s = fractional(f.coords, f.box)
    assert s.min() >= -1e-6 and s.max() < 1.0 + 1e-6  # wrapped into the cell
    sizes = np.diff(f.offsets)
    assert len(sizes) == 3 and sizes.sum() == 500_000 and sizes.max() - sizes.min() <= 1
    # clustered: 80 % of the particles in 200 clusters of sigma 2 give about 1/200 x
    # 0.64 of the pairs a same-cluster distance, half of them below 4 (about 3.7
    # times the close pairs of a uniform cell, ignoring images)
    rng = np.random.default_rng(0)
    idx = rng.choice(f.n, 4000, replace=False)
    d = np.linalg.norm(f.coords[idx][:, None, :] - f.coords[idx][None, :, :], axis=-1)
    close = (d[np.triu_indices(4000, 1)] < 4.0).mean()
    uniform = (4.0 / 3.0) * math.pi * 4.0 ** 3 / w.box_volume(f.box)
    assert close > 2 * uniform


def test_c4_batch():
    frames = w.batch_frames(seed=1)
    assert len(frames) == 256
    for f in frames:
        assert 5_000 <= f.n < 200_000 and f.box_type == w.BOX_ORTHO and f.nbins == 4096
        side = (f.n / 0.1) ** (1.0 / 3.0)
        assert np.allclose(w.box_matrix(f.box), np.diag([side] * 3))
        assert math.isclose(f.r_max, side / 2.0)
        assert list(f.offsets) == [0, int(round(0.3 * f.n)), f.n]
    ln = np.log([f.n for f in frames])  # log-uniform: mean near the middle of the log range
    assert abs(ln.mean() - 0.5 * (math.log(5_000) + math.log(200_000))) < 0.3


def test_c5_served_requests():
    rng = w.rng_for(2024)
    reqs = [w.served_request(rng) for _ in range(200)]
    assert {f.box_type for f in reqs} == {w.BOX_NONE, w.BOX_ORTHO, w.BOX_TRICLINIC}
    assert {len(f.offsets) - 1 for f in reqs} == {1, 2, 3}
    for f in reqs:
        assert 1_000 <= f.n < 1_000_000
        assert f.nbins in (1024, 2048, 4096, 8192, 16384)
        vol = f.n / 0.1
        if f.box_type == w.BOX_TRICLINIC:
            assert math.isclose(w.box_volume(f.box), vol, rel_tol=1e-9)
            assert math.isclose(f.r_max, 0.95 * float(w.box_heights(f.box).min()) / 2.0)
        else:
            side = vol ** (1.0 / 3.0)
            assert math.isclose(f.r_max, side / 2.0 if f.box_type == w.BOX_ORTHO else side * math.sqrt(3.0))


@pytest.mark.parametrize("box_type", [w.BOX_NONE, w.BOX_ORTHO, w.BOX_TRICLINIC])
def test_headline_frames(box_type):
    f = w.headline_frame(box_type, seed=11 + box_type, n=1_000_000)
    assert f.n == 1_000_000 and f.nbins == 10_000 and list(f.offsets) == [0, 1_000_000]
    assert f.n_pairs() == 499_999_500_000
    side = 1e7 ** (1.0 / 3.0)
    if box_type == w.BOX_TRICLINIC:
        assert math.isclose(w.box_volume(f.box), 1e7, rel_tol=1e-9)
        assert np.allclose(angles_of(f.box)[1], w.C3_ANGLES)
        assert math.isclose(f.r_max, 0.95 * float(w.box_heights(f.box).min()) / 2.0)
    else:
        assert abs(side - 215.44) < 0.01
        assert math.isclose(f.r_max, side / 2.0 if box_type == w.BOX_ORTHO else side * math.sqrt(3.0))
        assert f.coords.min() >= 0.0 and f.coords.max() < side


def test_generators_are_seeded():
    a, b = w.uniform_frame(5, 1000, w.BOX_ORTHO, w.ortho_box(10.0), 4.0, 100), \
        w.uniform_frame(5, 1000, w.BOX_ORTHO, w.ortho_box(10.0), 4.0, 100)
    c = w.uniform_frame(6, 1000, w.BOX_ORTHO, w.ortho_box(10.0), 4.0, 100)
    assert np.array_equal(a.coords, b.coords) and not np.array_equal(a.coords, c.coords)
    assert np.array_equal(w.config_small_nobox(seed=3).coords, w.config_small_nobox(seed=3).coords)
