"""Autotuned launch shapes (DH_CFG_AUTOTUNE, dh_config.tune_cache).

Every launch shape the autotuner may pick (j-tile length 256/512/1024, blocks
of 256, 512 or 1024 threads, one to eight histogram copies per block, blocks
per SM) must give the FP64 oracle's histogram bin for bin; the shapes are forced through the tuner's own
cache file.  The autotuner must measure each new launch key once, record it in
the file, and a context that reads the file must use it without measuring.
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


def sm_count(torch):
    return torch.cuda.get_device_properties(0).multi_processor_count


def variant_of(f):
    if f.box_type == w.BOX_NONE:
        return 0
    if f.box_type == w.BOX_ORTHO:
        return 1
    h_min = float(w.box_heights(f.box).min())
    return 2 if f.r_max <= (1.0 - 2.0 ** -8) * h_min / 2.0 else 3


def tune_key(frames):
    """The launch key of a batch of single-sweep frames of one variant."""
    width = max(f.nbins for f in frames)
    pairs = sum(f.n_pairs() for f in frames) / len(frames)
    wl = max(0, math.ceil(math.log2(width)))
    nl = math.floor(math.log2(math.sqrt(2.0 * max(pairs, 1.0))) + 0.5)
    f4 = 0
    while f4 < 3 and (1 << (2 * (f4 + 1))) <= len(frames):
        f4 += 1
    return variant_of(frames[0]), wl, nl, f4


def write_cache(path, sms, keys, tile_j, depth, bps, block=256, agg=None):
    lines = ["# forced shapes"]
    for v, wl, nl, f4 in keys:
        tail = "" if agg is None else f" {agg}"
        lines.append(f"{sms} {v} {wl} {nl} {f4} {tile_j} {block} {depth} {bps} 1.0{tail}")
    path.write_text("\n".join(lines) + "\n")


def device_args(torch, frames):
    return [dh.FrameArgs(torch.from_numpy(f.coords).cuda(), f.offsets, f.box_type, f.box, f.r_max, f.nbins)
            for f in frames]


def result(fa):
    return fa.out.cpu().numpy().view(np.uint64)


TRIC = w.triclinic_box(20, 20, 20, *w.C3_ANGLES)
FRAMES = {
    "nobox_ragged": w.uniform_frame(31, 3001, w.BOX_NONE, w.ortho_box(9.0), 16.0, 1000),
    "ortho_3species": w.frame_from(w.uniform_frame(32, 4200, w.BOX_ORTHO, w.ortho_box(24.0), 11.0, 5000).coords,
                                   [0, 1000, 3500, 4200], w.BOX_ORTHO, w.ortho_box(24.0), 11.0, 5000, "o3"),
    "tric_2species": w.uniform_frame(33, 2600, w.BOX_TRICLINIC, TRIC, 9.0, 3000, n_species=2),
    "tric_search": w.uniform_frame(34, 1500, w.BOX_TRICLINIC, TRIC, 14.0, 2000),
}
SHAPES = [(256, 1, 3, 256), (512, 2, 2, 256), (256, 4, 1, 256), (1024, 2, 3, 256), (512, 4, 2, 256),
          (1024, 1, 1, 256), (1024, 1, 1, 512), (256, 2, 1, 512), (512, 4, 1, 512), (1024, 1, 1, 1024),
          (256, 2, 1, 1024), (1024, 8, 1, 256), (512, 8, 1, 1024), (1024, 4, 1, 1024)]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"tj{s[0]}_d{s[1]}_b{s[2]}_t{s[3]}")
def test_forced_shapes_match_oracle(torch_mod, oracle_mod, tmp_path, shape):
    tile_j, depth, bps, block = shape
    sms = sm_count(torch_mod)
    path = tmp_path / "tune.txt"
    write_cache(path, sms, [tune_key([f]) for f in FRAMES.values()], tile_j, depth, bps, block)
    assert dh.dh_tune_cache_count(str(path), sms) == len(FRAMES)
    with dh.Context(0, tune_cache=str(path)) as ctx:
        for name, f in FRAMES.items():
            x = torch_mod.from_numpy(f.coords).cuda()
            got = ctx.histogram(x, f.offsets, f.box_type, f.box, f.r_max, f.nbins).cpu().numpy().view(np.uint64)
            st = ctx.stats()
            assert (st["tile_j"], st["hist_depth"], st["block_threads"]) == (tile_j, depth, block), name
            assert 1 <= st["blocks_per_sm"] <= bps
            assert st["tune_runs"] == 0
            assert np.array_equal(got, oracle_mod.histogram_frame(f)), name


@pytest.mark.parametrize("tile_j", [1024, 256])
def test_forced_warp_aggregated_increments(torch_mod, oracle_mod, tmp_path, tile_j):
    # the lanes of a warp that hit one bin add their count once (match.any);
    # every variant, masked diagonal tiles and ragged tails
    sms = sm_count(torch_mod)
    path = tmp_path / "tune.txt"
    write_cache(path, sms, [tune_key([f]) for f in FRAMES.values()], tile_j, 1, 3, 256, agg=1)
    with dh.Context(0, tune_cache=str(path)) as ctx:
        for name, f in FRAMES.items():
            x = torch_mod.from_numpy(f.coords).cuda()
            got = ctx.histogram(x, f.offsets, f.box_type, f.box, f.r_max, f.nbins).cpu().numpy().view(np.uint64)
            st = ctx.stats()
            assert st["warp_agg"] == 1 and st["block_threads"] == 256 and st["tile_j"] == tile_j, name
            assert np.array_equal(got, oracle_mod.histogram_frame(f)), name
        # clustered bins: a small cube whose pairs share few bins
        g = w.frame_from((w.rng_for(37).random((5000, 3)) * 2.0).astype(np.float32), [0, 5000], w.BOX_NONE,
                         np.zeros(9), 3.5, 40, "clustered")
        write_cache(path, sms, [tune_key([g])], tile_j, 1, 3, 256, agg=1)
    with dh.Context(0, tune_cache=str(path)) as ctx:
        got = ctx.histogram(torch_mod.from_numpy(g.coords).cuda(), g.offsets, g.box_type, g.box, g.r_max,
                            g.nbins).cpu().numpy().view(np.uint64)
        assert ctx.stats()["warp_agg"] == 1
        assert np.array_equal(got, oracle_mod.histogram_frame(g))


def test_forced_shape_multi_sweep(torch_mod, oracle_mod, tmp_path):
    # wider than shared memory: several bin sweeps (the histogram width key is the sweep width)
    f = w.uniform_frame(35, 2500, w.BOX_ORTHO, w.ortho_box(12.0), 6.0, 150_000, n_species=2)
    sms = sm_count(torch_mod)
    v, _, nl, f4 = tune_key([f])
    path = tmp_path / "tune.txt"
    write_cache(path, sms, [(v, wl, nl, f4) for wl in range(14, 18)], 512, 2, 2, 512)
    with dh.Context(0, tune_cache=str(path)) as ctx:
        x = torch_mod.from_numpy(f.coords).cuda()
        got = ctx.histogram(x, f.offsets, f.box_type, f.box, f.r_max, f.nbins).cpu().numpy().view(np.uint64)
        st = ctx.stats()
        assert st["sweeps"] >= 2 and st["tile_j"] == 512 and st["block_threads"] in (256, 512, 1024)
        assert np.array_equal(got, oracle_mod.histogram_frame(f))


def test_autotune_measures_once_and_reuses_the_file(torch_mod, oracle_mod, tmp_path):
    frames = w.batch_frames(seed=36, n_frames=20, n_lo=500, n_hi=6000)
    path = tmp_path / "tune.txt"
    sms = sm_count(torch_mod)
    flags = dh.DH_CFG_AUTOTUNE | dh.DH_CFG_TIMING
    with dh.Context(0, flags=flags, tune_cache=str(path)) as ctx:
        fas = device_args(torch_mod, frames)
        ctx.histogram_batch(fas)
        st = ctx.stats()
        assert st["tune_runs"] > 1
        shape = (st["tile_j"], st["hist_depth"], st["blocks_per_sm"], st["block_threads"])
        assert shape[0] in (256, 512, 1024) and shape[1] in (1, 2, 4) and shape[2] >= 1
        assert shape[3] in (256, 512, 1024)
        for fa, f in zip(fas, frames):
            assert np.array_equal(result(fa), oracle_mod.histogram_frame(f)), f.name
        ctx.histogram_batch(fas)  # same key: no new measurement
        assert ctx.stats()["tune_runs"] == 0
    assert dh.dh_tune_cache_count(str(path), sms) >= 1
    with dh.Context(0, flags=flags, tune_cache=str(path)) as ctx:
        fas2 = device_args(torch_mod, frames)
        ctx.histogram_batch(fas2)
        st = ctx.stats()
        assert st["tune_runs"] == 0
        assert (st["tile_j"], st["hist_depth"], st["blocks_per_sm"], st["block_threads"]) == shape
        for fa, fb in zip(fas, fas2):
            assert np.array_equal(result(fa), result(fb))
