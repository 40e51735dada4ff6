"""The float32 decision rule against its own error analysis, on the GPU.

The fast path decides a pair in float32 only when its bin coordinate t lies
farther than delta from every integer; delta is derived per frame from the
operation sequence.  These checks measure, on sampled pairs at full size, how
much of delta the actual error uses (must stay below 1) and count pairs whose
float32 decision would differ from the binary64 definition (must be 0).
"""
import numpy as np
import pytest

import paper_1808_01478_gb300 as dh
import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = dh.Context(0)
    yield c
    c.close()


def test_sqrt_approx_within_assumed_bound(ctx):
    err = ctx.check_sqrt()
    assert 0.0 < err <= 2.0 ** -21, err


FRAMES = {
    "ortho_c2": lambda: w.config_ortho_two_species(seed=1),
    "tric_c3": lambda: w.config_triclinic_clusters(seed=1),
    "nobox_c1": lambda: w.config_small_nobox(seed=1),
    "headline_none": lambda: w.headline_frame(w.BOX_NONE, seed=11),
    "headline_ortho": lambda: w.headline_frame(w.BOX_ORTHO, seed=12),
    "headline_tric": lambda: w.headline_frame(w.BOX_TRICLINIC, seed=13),
    "tric_search": lambda: w.uniform_frame(6, 50000, w.BOX_TRICLINIC, w.triclinic_box(20, 20, 20, *w.C3_ANGLES),
                                           14.0, 2000),
    "wide_bins": lambda: w.uniform_frame(9, 100000, w.BOX_ORTHO, w.ortho_box(40.0), 20.0, 150_000),
}


@pytest.mark.parametrize("name", sorted(FRAMES))
def test_window_bound_holds(ctx, name):
    f = FRAMES[name]()
    res = ctx.check_window(f.coords, f.offsets, f.box_type, f.box, f.r_max, f.nbins, n_samples=1 << 23, seed=7)
    assert res["checked"] > 1 << 20
    assert res["violations"] == 0, res
    assert res["max_ratio"] < 1.0, res


TILE_FRAMES = {
    "ortho_c2": lambda: w.config_ortho_two_species(seed=1),
    "tric_c3": lambda: w.config_triclinic_clusters(seed=1),
    "headline_ortho": lambda: w.headline_frame(w.BOX_ORTHO, seed=12),
    "headline_tric": lambda: w.headline_frame(w.BOX_TRICLINIC, seed=13),
    "ortho_small_box": lambda: w.uniform_frame(17, 60000, w.BOX_ORTHO, w.ortho_box(30.0, 26.0, 34.0), 12.9, 4000),
}


@pytest.mark.parametrize("name", sorted(TILE_FRAMES))
def test_tile_mode_windows_hold(ctx, name):
    # every pair of sampled warp tiles, in the tile's image mode with its own
    # window (uniform, one axis wrapped, or per pair), against binary64
    f = TILE_FRAMES[name]()
    res = ctx.check_tiles(f.coords, f.offsets, f.box_type, f.box, f.r_max, f.nbins, n_tiles=4096, seed=9)
    assert res["checked"] > 1 << 24
    assert res["shifted_tiles"] > 0, res
    assert res["violations"] == 0, res
    assert res["max_ratio"] < 1.0, res


def test_tile_check_rejects_other_boxes(ctx):
    f = w.config_small_nobox(seed=1)
    with pytest.raises(dh.DHError) as e:
        ctx.check_tiles(f.coords, f.offsets, f.box_type, f.box, f.r_max, f.nbins)
    assert e.value.status == dh.DH_ERR_INVALID


def _f64(f):
    # the same frame with binary64 coordinates that are not float32 values
    x = f.coords.astype(np.float64) + w.rng_for(5).random(f.coords.shape) * 1e-5
    return x, f


F64_FRAMES = {
    "f64_ortho": lambda: _f64(w.headline_frame(w.BOX_ORTHO, seed=14, n=300_000)),
    "f64_tric": lambda: _f64(w.headline_frame(w.BOX_TRICLINIC, seed=15, n=300_000)),
    "f64_none": lambda: _f64(w.headline_frame(w.BOX_NONE, seed=16, n=300_000)),
}


@pytest.mark.parametrize("name", sorted(F64_FRAMES))
def test_window_bound_holds_for_binary64_input(ctx, name):
    x, f = F64_FRAMES[name]()
    res = ctx.check_window(x, f.offsets, f.box_type, f.box, f.r_max, f.nbins, n_samples=1 << 23, seed=8)
    assert res["checked"] > 1 << 20
    assert res["violations"] == 0, res
    assert res["max_ratio"] < 1.0, res
