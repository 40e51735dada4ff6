"""Seeded random frames against the FP64 oracle, bin for bin.

Each frame draws its box type, a reduced triclinic cell or an orthorhombic box
of random shape, r_max on either side of half the smallest plane spacing (the
one-wrap and the 27-image-search variants), the bin count, the species split
(empty and one-particle species included), the coordinate scale, an offset
far from the origin and unwrapping by whole cells, and float32 or binary64
coordinates.  The frames are small, so the oracle decides them in well under a
second each; together they reach every minimum-image variant, the spatial
order, the tile images and culling, several bin sweeps and the deferral tiers.
"""
import math

import numpy as np
import pytest

import paper_1808_01478_gb300 as dh
import workloads as w

pytestmark = pytest.mark.gpu

N_FRAMES = 60


@pytest.fixture(scope="module")
def torch_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def reduced_triclinic(rng, scale):
    """An upper-triangular cell with |bx|, |cx| <= ax/2 and |cy| <= by/2."""
    ax, by, cz = scale * (0.7 + 0.6 * rng.random(3))
    bx = (rng.random() - 0.5) * ax
    cx = (rng.random() - 0.5) * ax
    cy = (rng.random() - 0.5) * by
    return np.array([ax, bx, cx, 0.0, by, cy, 0.0, 0.0, cz])


def random_frame(k):
    rng = w.rng_for(9000 + k)
    box_type = int(rng.integers(0, 3))
    scale = float(10.0 ** rng.uniform(-1.0, 3.0))
    n = int(rng.integers(2, 2600))
    n_species = int(rng.integers(1, 5))
    cuts = np.sort(rng.integers(0, n + 1, size=n_species - 1))
    offsets = np.concatenate([[0], cuts, [n]]).astype(np.int64)
    nbins = int(rng.choice([1, 7, 64, 1000, 4096, 20000, 70000]))
    if box_type == w.BOX_NONE:
        box = np.zeros(9)
        x = rng.random((n, 3)) * scale
        diag = scale * math.sqrt(3.0)
        r_max = diag * float(rng.choice([0.3, 0.7, 1.01, 2.0]))
    else:
        box = reduced_triclinic(rng, scale) if box_type == w.BOX_TRICLINIC else w.ortho_box(*(scale * (0.7 + 0.6 * rng.random(3))))
        m = w.box_matrix(box)
        x = (m @ rng.random((n, 3)).T).T
        h = float(w.box_heights(box).min())
        r_max = h * float(rng.choice([0.2, 0.45, 0.49, 0.7]))
        if rng.random() < 0.3:  # unwrapped by whole cells
            x = x + (rng.integers(-50, 51, size=(n, 3)).astype(np.float64) @ m.T)
    if rng.random() < 0.2:  # far from the origin
        x = x + 1000.0 * scale
    f64 = bool(rng.random() < 0.25)
    x = np.ascontiguousarray(x, dtype=np.float64 if f64 else np.float32)
    return x, offsets, box_type, box, r_max, nbins


@pytest.mark.parametrize("k", range(N_FRAMES))
def test_random_frame_matches_oracle(torch_mod, oracle_mod, k):
    x, offs, box_type, box, r_max, nbins = random_frame(k)
    want = oracle_mod.histogram(x, offs, box_type, box, r_max, nbins)
    with dh.Context(0) as ctx:
        got = ctx.histogram(torch_mod.from_numpy(x).cuda(), offs, box_type, box, r_max, nbins)
    got = got.cpu().numpy().view(np.uint64)
    assert got.shape == want.shape
    bad = np.argwhere(got != want)
    assert bad.size == 0, (k, box_type, x.dtype, x.shape[0], nbins, r_max, len(bad), bad[:3].tolist())


def test_random_frames_batched(torch_mod, oracle_mod):
    # the same generator through dh_histogram_batch (one persistent launch per
    # variant present, replayed as a CUDA graph), 12 frames per call
    frames = [random_frame(k) for k in range(500, 524)]
    with dh.Context(0) as ctx:
        for b in range(0, len(frames), 12):
            chunk = frames[b:b + 12]
            fas = [dh.FrameArgs(torch_mod.from_numpy(x).cuda(), o, bt, bx, r, nb) for (x, o, bt, bx, r, nb) in chunk]
            ctx.histogram_batch(fas)
            assert ctx.stats()["graph_replays"] == 1
            for q, (fa, f) in enumerate(zip(fas, chunk)):
                got = fa.out.cpu().numpy().view(np.uint64)
                assert np.array_equal(got, oracle_mod.histogram(*f)), b + q
