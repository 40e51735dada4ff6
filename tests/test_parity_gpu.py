"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, bin for bin.

Histogram counts are integers, so the bar is bit-exact equality on every bin.
Sizes are chosen so the oracle finishes in seconds while the GPU work still
spans several 1024x1024 tiles with ragged tails.
"""
import math

import numpy as np
import pytest

import paper_1808_01478_gb300 as dh
import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def ctx(torch_mod):
    c = dh.Context(0)
    yield c
    c.close()


def gpu_hist(ctx, torch, f, device=True, f4=False):
    if device:
        x = torch.from_numpy(f.coords).cuda()
        if f4:
            x = torch.cat([x, torch.zeros_like(x[:, :1])], 1).contiguous()
        out = ctx.histogram(x, f.offsets, f.box_type, f.box, f.r_max, f.nbins)
        torch.cuda.synchronize()
        return out.cpu().numpy().view(np.uint64)
    c = f.coords
    if f4:
        c = np.concatenate([c, np.zeros((c.shape[0], 1), np.float32)], 1)
    return ctx.histogram(c, f.offsets, f.box_type, f.box, f.r_max, f.nbins)


def assert_same(got, want, name=""):
    assert got.shape == want.shape, (got.shape, want.shape)
    if not np.array_equal(got, want):
        bad = np.argwhere(got != want)
        h, k = bad[0]
        raise AssertionError(f"{name}: {len(bad)} bins differ; first (h={h}, bin={k}): "
                             f"gpu {got[h, k]} oracle {want[h, k]}; sums {got.sum()} vs {want.sum()}")


def small_cases():
    tric = w.triclinic_box(80, 80, 80, *w.C3_ANGLES)
    return {
        "nobox_c1": w.config_small_nobox(seed=1),
        "nobox_ragged": w.uniform_frame(4, 3333, w.BOX_NONE, w.ortho_box(9.0), 16.0, 1000),
        "ortho_c2_small": w.config_ortho_two_species(seed=2, n=6000),
        "ortho_aniso": w.uniform_frame(5, 4100, w.BOX_ORTHO, w.ortho_box(20.0, 13.0, 31.0), 6.4, 3000,
                                       n_species=3),
        "tric_c3_small": w.config_triclinic_clusters(seed=3, n=6000, n_clusters=10, edge=80.0),
        "tric_search": w.uniform_frame(6, 2500, w.BOX_TRICLINIC, w.triclinic_box(20, 20, 20, *w.C3_ANGLES),
                                       14.0, 2000, n_species=2),
        "tric_skewed": w.uniform_frame(7, 3000, w.BOX_TRICLINIC, w.triclinic_box(30, 25, 28, 80, 75, 105),
                                       0.9 * w.box_heights(w.triclinic_box(30, 25, 28, 80, 75, 105)).min() / 2,
                                       5000),
        "tric_c3_box_uniform": w.uniform_frame(8, 4000, w.BOX_TRICLINIC, tric, 35.0, 20000, n_species=3),
    }


CASES = small_cases()


@pytest.mark.parametrize("name", sorted(CASES))
def test_parity_small(ctx, torch_mod, oracle_mod, name):
    f = CASES[name]
    want = oracle_mod.histogram_frame(f)
    got = gpu_hist(ctx, torch_mod, f)
    assert_same(got, want, name)
    st = ctx.stats()
    assert st["pairs"] == f.n_pairs()


@pytest.mark.parametrize("name", ["nobox_ragged", "ortho_c2_small", "tric_c3_small"])
def test_parity_host_pointers_and_f4(ctx, torch_mod, oracle_mod, name):
    f = CASES[name]
    want = oracle_mod.histogram_frame(f)
    assert_same(gpu_hist(ctx, torch_mod, f, device=False), want, name + "/host")
    assert_same(gpu_hist(ctx, torch_mod, f, device=True, f4=True), want, name + "/f4")
    assert_same(gpu_hist(ctx, torch_mod, f, device=False, f4=True), want, name + "/host-f4")


def test_multi_sweep_wide_histogram(ctx, torch_mod, oracle_mod):
    # more bins than one block's shared memory holds: several passes over the pairs
    f = w.uniform_frame(9, 3000, w.BOX_ORTHO, w.ortho_box(40.0), 20.0, 150_000, n_species=2)
    want = oracle_mod.histogram_frame(f)
    got = gpu_hist(ctx, torch_mod, f)
    assert ctx.stats()["sweeps"] >= 2
    assert_same(got, want, "multi-sweep")


@pytest.mark.parametrize("spacing,box_type", [(0.1, w.BOX_NONE), (0.25, w.BOX_ORTHO), (0.5, w.BOX_NONE)])
def test_adversarial_lattice_edges(ctx, torch_mod, oracle_mod, spacing, box_type):
    # lattice spacing == bin width: a large share of pairs sits within ulps of bin edges
    per = 14
    g = np.arange(per, dtype=np.float64) * spacing
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).astype(np.float32)
    side = per * spacing
    if box_type == w.BOX_ORTHO:
        box = w.ortho_box(side)
        r_max = side / 2
    else:
        box = np.zeros(9)
        r_max = side * math.sqrt(3)
    nbins = int(round(r_max / spacing))
    f = w.frame_from(x, [0, len(x)], box_type, box, r_max, nbins, "lattice")
    want = oracle_mod.histogram_frame(f)
    got = gpu_hist(ctx, torch_mod, f)
    assert_same(got, want, "lattice")
    assert ctx.stats()["deferred"] > 0


def test_edge_sizes(ctx, torch_mod, oracle_mod):
    rng = np.random.default_rng(0)
    for n, offs in [(0, [0, 0]), (1, [0, 1]), (2, [0, 2]), (5, [0, 0, 5, 5]), (1025, [0, 1, 1024, 1025]),
                    (2049, [0, 2049]), (1024, [0, 512, 1024])]:
        x = (rng.random((n, 3)) * 5).astype(np.float32)
        f = w.frame_from(x, offs, w.BOX_NONE, np.zeros(9), 9.0, 17, f"n{n}")
        want = oracle_mod.histogram_frame(f)
        got = ctx.histogram(x, offs, f.box_type, f.box, f.r_max, f.nbins)
        assert_same(got, want, f.name)
    # one bin, and more bins than pairs
    f = w.uniform_frame(1, 700, w.BOX_ORTHO, w.ortho_box(5.0), 2.5, 1)
    assert_same(gpu_hist(ctx, torch_mod, f), oracle_mod.histogram_frame(f), "nbins=1")


def test_accumulate(ctx, torch_mod, oracle_mod):
    f = CASES["ortho_aniso"]
    want = oracle_mod.histogram_frame(f)
    out = np.full(want.shape, 7, dtype=np.uint64)
    ctx.histogram(f.coords, f.offsets, f.box_type, f.box, f.r_max, f.nbins, out=out, accumulate=True)
    assert_same(out, want + np.uint64(7), "accumulate-host")
    x = torch_mod.from_numpy(f.coords).cuda()
    o = torch_mod.from_numpy(want.view(np.int64).copy()).cuda()
    ctx.histogram(x, f.offsets, f.box_type, f.box, f.r_max, f.nbins, out=o, accumulate=True)
    assert_same(o.cpu().numpy().view(np.uint64), want * np.uint64(2), "accumulate-device")


def test_invalid_arguments(ctx, torch_mod):
    x = np.zeros((4, 3), np.float32)
    x[2, 1] = np.nan
    with pytest.raises(dh.DHError) as e:
        ctx.histogram(x, [0, 4], w.BOX_NONE, None, 1.0, 4)
    assert e.value.status == dh.DH_ERR_INVALID
    good = np.random.default_rng(1).random((10, 3)).astype(np.float32)
    bad_cases = [
        dict(offsets=[0, 5], box_type=w.BOX_NONE, box=None, r_max=1.0, nbins=4),
        dict(offsets=[0, 10], box_type=w.BOX_NONE, box=None, r_max=-1.0, nbins=4),
        dict(offsets=[0, 10], box_type=w.BOX_NONE, box=None, r_max=1.0, nbins=0),
        dict(offsets=[0, 10], box_type=w.BOX_ORTHO, box=[1, 0.1, 0, 0, 1, 0, 0, 0, 1], r_max=1.0, nbins=4),
        dict(offsets=[0, 10], box_type=w.BOX_TRICLINIC, box=[1, 0.9, 0, 0, 1, 0, 0, 0, 1], r_max=0.1, nbins=4),
        dict(offsets=[0, 10], box_type=w.BOX_TRICLINIC, box=[1, 0, 0, 0.2, 1, 0, 0, 0, 1], r_max=0.1, nbins=4),
        dict(offsets=[0, 6, 4, 10], box_type=w.BOX_NONE, box=None, r_max=1.0, nbins=4),
        dict(offsets=[0, 10], box_type=7, box=None, r_max=1.0, nbins=4),
    ]
    for kw in bad_cases:
        with pytest.raises(dh.DHError) as e:
            ctx.histogram(good, **kw)
        assert e.value.status == dh.DH_ERR_INVALID, kw
    # the context stays usable after errors
    f = CASES["nobox_c1"]
    got = ctx.histogram(f.coords, f.offsets, f.box_type, f.box, f.r_max, f.nbins)
    assert int(got.sum()) == 1_999_000


def test_repeat_calls_identical_and_threshold_cache(ctx, torch_mod, oracle_mod):
    f = CASES["tric_c3_small"]
    want = oracle_mod.histogram_frame(f)
    for _ in range(3):
        assert_same(gpu_hist(ctx, torch_mod, f), want, "repeat")


# Species of periodic frames are put in spatial order before the pair kernel,
# and tile pairs whose float32 nearest images are provably the same for every
# pair (on all axes, or on all but one) skip the per-pair rounding of those
# axes; both must leave every bin unchanged.
SPATIAL = {
    "ortho_sorted_species": w.frame_from(
        w.uniform_frame(61, 30000, w.BOX_ORTHO, w.ortho_box(60.0, 50.0, 70.0), 25.0, 6000).coords,
        [0, 1500, 21000, 30000], w.BOX_ORTHO, w.ortho_box(60.0, 50.0, 70.0), 25.0, 6000, "ortho_sorted"),
    "tric_sorted": w.uniform_frame(62, 24000, w.BOX_TRICLINIC, w.triclinic_box(64, 64, 64, *w.C3_ANGLES),
                                   28.0, 8000, n_species=2),
    "ortho_unwrapped": w.frame_from(
        (w.uniform_frame(63, 12000, w.BOX_ORTHO, w.ortho_box(40.0), 19.0, 3000).coords
         + np.float32(40.0) * w.rng_for(64).integers(-2, 3, size=(12000, 3)).astype(np.float32)),
        [0, 12000], w.BOX_ORTHO, w.ortho_box(40.0), 19.0, 3000, "ortho_unwrapped"),
}


@pytest.mark.parametrize("name", sorted(SPATIAL))
def test_spatial_order_and_tile_images(ctx, torch_mod, oracle_mod, name):
    f = SPATIAL[name]
    got = gpu_hist(ctx, torch_mod, f)
    assert_same(got, oracle_mod.histogram_frame(f), name)
    st = ctx.stats()
    if name == "ortho_sorted_species":
        assert st["uniform_pairs"] > 0 and st["axis_pairs"] > 0, st
    assert st["uniform_pairs"] + st["axis_pairs"] <= st["pairs"]


@pytest.mark.parametrize("box_type", [w.BOX_ORTHO, w.BOX_TRICLINIC])
def test_tile_images_at_larger_n_match_the_unsorted_path(ctx, torch_mod, oracle_mod, box_type):
    # N = 131,072: the sorted path with tile images against dh_histogram_noalloc,
    # which does not sort (its warps see unsorted runs, which rarely share one
    # nearest image), bin for bin; and, independently, the histograms of a
    # species of 2,048 particles carved out of the same frame (its AA and AB
    # pairs against every particle) against the oracle
    n = dh.DH_NOALLOC_MAX_N
    if box_type == w.BOX_ORTHO:
        box = w.ortho_box((n / 0.1) ** (1.0 / 3.0))
        r_max = box[0] / 2.0
    else:
        box = w.scale_box(w.triclinic_box(1.0, 1.0, 1.0, *w.C3_ANGLES), n / 0.1)
        r_max = 0.95 * float(w.box_heights(box).min()) / 2.0
    f = w.uniform_frame(65, n, box_type, box, r_max, 10_000)
    x = torch_mod.from_numpy(f.coords).cuda()
    got = ctx.histogram(x, f.offsets, f.box_type, f.box, f.r_max, f.nbins).cpu().numpy().view(np.uint64)
    st = ctx.stats()
    assert 0 < st["uniform_pairs"] <= st["pairs"], st
    assert 0 < st["axis_pairs"] <= st["pairs"] - st["uniform_pairs"], st  # one-axis tiles exercised too
    out = torch_mod.zeros((1, f.nbins), dtype=torch_mod.int64, device="cuda")
    fa = dh.FrameArgs(x, f.offsets, f.box_type, f.box, f.r_max, f.nbins, out)
    dh.dh_histogram_noalloc(fa.frame)
    assert_same(got, out.cpu().numpy().view(np.uint64), "noalloc")
    g = w.frame_from(f.coords, [0, 2048, n], f.box_type, f.box, f.r_max, f.nbins, "carved")
    h = ctx.histogram(x, g.offsets, g.box_type, g.box, g.r_max, g.nbins).cpu().numpy().view(np.uint64)
    assert ctx.stats()["uniform_pairs"] > 0
    for k, (a, c) in enumerate([(0, 0), (0, 1)]):
        want = oracle_mod.histogram_one(g.coords, g.offsets, g.box_type, g.box, g.r_max, g.nbins, a, c)
        assert np.array_equal(h[k], want), (a, c)
    assert np.array_equal(h.sum(0), got[0])  # the split histograms add up to the frame's


@pytest.mark.parametrize("box_type,n,nbins", [(w.BOX_ORTHO, 40000, 150_000), (w.BOX_TRICLINIC, 30000, 120_000),
                                              (w.BOX_ORTHO, 60000, 10_000), (w.BOX_NONE, 40000, 150_000),
                                              (w.BOX_NONE, 50000, 5_000)])
def test_tiles_outside_the_sweep_are_skipped(ctx, torch_mod, oracle_mod, box_type, n, nbins):
    # spatially sorted periodic frames at density 0.1: warp tiles whose distance
    # bounds put no pair in the current bin sweep (or beyond r_max) are skipped;
    # several sweeps, and one, against the oracle bin for bin
    if box_type == w.BOX_NONE:  # a cube, r_max its diagonal (several sweeps) or a fifth of it (one)
        side = (n / 0.1) ** (1.0 / 3.0)
        r_max = side * math.sqrt(3.0) * (1.0 if nbins > 100_000 else 0.2)
        g = w.uniform_frame(66, n, w.BOX_ORTHO, w.ortho_box(side), r_max, nbins, n_species=2)
        f = w.frame_from(g.coords, g.offsets, w.BOX_NONE, np.zeros(9), r_max, nbins, "nobox-cull")
    else:
        if box_type == w.BOX_ORTHO:
            box = w.ortho_box((n / 0.1) ** (1.0 / 3.0))
            r_max = box[0] / 2.0
        else:
            box = w.scale_box(w.triclinic_box(1.0, 1.0, 1.0, *w.C3_ANGLES), n / 0.1)
            r_max = 0.95 * float(w.box_heights(box).min()) / 2.0
        f = w.uniform_frame(66, n, box_type, box, r_max, nbins, n_species=2)
    got = gpu_hist(ctx, torch_mod, f)
    st = ctx.stats()
    assert st["culled_pairs"] > 0, st
    if nbins > 100_000:
        assert st["sweeps"] >= 2, st
    assert_same(got, oracle_mod.histogram_frame(f), f"cull-{n}-{nbins}")


@pytest.mark.parametrize("cells", [3000, 40000])
def test_far_unwrapped_triclinic_coordinates(ctx, torch_mod, oracle_mod, cells):
    # particles of a 20 A triclinic cell moved by random lattice vectors of up to
    # `cells` cells (unwrapped trajectories): the coordinate ranges are so wide
    # that the float32 nearest images cannot be trusted, so every pair is
    # decided without them; r_max just below half the smallest plane spacing
    box = w.triclinic_box(20, 20, 20, *w.C3_ANGLES)
    h = float(w.box_heights(box).min())
    f0 = w.uniform_frame(67, 1500, w.BOX_TRICLINIC, box, 0.99 * h / 2.0, 800, n_species=2)
    k = w.rng_for(68).integers(-cells, cells + 1, size=(f0.n, 3)).astype(np.float64)
    x = (f0.coords.astype(np.float64) + k @ w.box_matrix(box).T).astype(np.float32)
    f = w.frame_from(x, f0.offsets, f0.box_type, f0.box, f0.r_max, f0.nbins, f"tric-unwrapped-{cells}")
    assert_same(gpu_hist(ctx, torch_mod, f), oracle_mod.histogram_frame(f), f.name)


@pytest.mark.parametrize("cells", [3000, 200000, 3000000])
def test_far_unwrapped_orthorhombic_coordinates(ctx, torch_mod, oracle_mod, cells):
    box = w.ortho_box(20.0, 17.0, 23.0)
    f0 = w.uniform_frame(69, 1500, w.BOX_ORTHO, box, 8.4, 800, n_species=2)
    k = w.rng_for(70).integers(-cells, cells + 1, size=(f0.n, 3)).astype(np.float64)
    x = (f0.coords.astype(np.float64) + k * np.array([20.0, 17.0, 23.0])).astype(np.float32)
    f = w.frame_from(x, f0.offsets, f0.box_type, f0.box, f0.r_max, f0.nbins, f"ortho-unwrapped-{cells}")
    assert_same(gpu_hist(ctx, torch_mod, f), oracle_mod.histogram_frame(f), f.name)


def test_far_offset_no_box(ctx, torch_mod, oracle_mod):
    # a compact cluster far from the origin: differences of large, close coordinates
    rng = w.rng_for(71)
    x = (1.0e6 + rng.random((2500, 3)) * 30.0).astype(np.float32)
    f = w.frame_from(x, [0, 1200, 2500], w.BOX_NONE, np.zeros(9), 40.0, 3000, "nobox-offset")
    assert_same(gpu_hist(ctx, torch_mod, f), oracle_mod.histogram_frame(f), f.name)


@pytest.mark.parametrize("box_type,cells", [(w.BOX_TRICLINIC, 5000), (w.BOX_ORTHO, 100000)])
def test_far_unwrapped_binary64_input(ctx, torch_mod, oracle_mod, box_type, cells):
    # binary64 coordinates (all 53 bits used) spread over many cells
    if box_type == w.BOX_TRICLINIC:
        box = w.triclinic_box(20, 20, 20, *w.C3_ANGLES)
        r_max = 0.95 * float(w.box_heights(box).min()) / 2.0
    else:
        box = w.ortho_box(20.0, 17.0, 23.0)
        r_max = 8.4
    rng = w.rng_for(72)
    m = w.box_matrix(box)
    x = (m @ rng.random((1500, 3)).T).T
    x = x + (rng.integers(-cells, cells + 1, size=(1500, 3)).astype(np.float64) @ m.T)
    offs = w.even_offsets(1500, 2)
    want = oracle_mod.histogram(x, offs, box_type, box, r_max, 700)
    got = ctx.histogram(torch_mod.from_numpy(x).cuda(), offs, box_type, box, r_max, 700)
    assert_same(got.cpu().numpy().view(np.uint64), want, "f64-unwrapped")


@pytest.mark.parametrize("box_type", [w.BOX_ORTHO, w.BOX_TRICLINIC])
def test_half_box_ties_on_a_lattice(ctx, torch_mod, oracle_mod, box_type):
    # an integer lattice in a box of side 16: many displacements are exactly
    # L/2 = 8 on one or more axes, where the nearest image of Eq. 5 is a tie
    # (half to even in binary64 and in float32); r_max beyond L/2 (orthorhombic)
    # and beyond half the plane spacing (triclinic: the 27-image search)
    g = np.arange(16, dtype=np.float32)
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)[::3].copy()
    if box_type == w.BOX_ORTHO:
        box, r_max, nbins = w.ortho_box(16.0), 12.0, 48
    else:
        box = np.array([16.0, 4.0, 2.0, 0.0, 16.0, 4.0, 0.0, 0.0, 16.0])
        r_max, nbins = 10.0, 40
    f = w.frame_from(x, [0, 600, x.shape[0]], box_type, box, r_max, nbins, "half-box-ties")
    got = gpu_hist(ctx, torch_mod, f)
    assert ctx.stats()["deferred"] > 0
    assert_same(got, oracle_mod.histogram_frame(f), f.name)
