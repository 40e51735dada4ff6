"""The tiers that decide exactness, each shown to run and to agree with the oracle.

Bit-exactness against the binary64 definition (Alg. 1 with the half-open bins
of Eq. 4 and the minimum image of Eq. 5) rests on three mechanisms the common
inputs rarely reach:

* the binary64 replay of a deferred pair, reached only when even the
  double-float tier cannot tell r^2 from a binary64 bin threshold (about one
  deferred pair in 10^4 on random inputs).  Integer lattices with a dyadic bin
  width put many pairs exactly on a threshold: r = k dr, so r^2 = T[k] and the
  double-float difference is zero.  Each minimum-image variant (no box,
  orthorhombic, triclinic below half the plane spacing with its m = 0
  shortcut, triclinic with the 27-image search) and binary64 input must show
  ``exact_fallback > 0`` and equal the oracle bin for bin;
* the flush of a block's uint32 shared-memory counts into the uint64 global
  histogram before 2^32 pairs accumulate (the paper's flush of 32-bit private
  counts, Sec. 3.1): one block per SM over 2*10^12 pairs puts about 9*10^9
  pairs of one bin into each block;
* full-size C2 and C3 and the 256-frame C4 batch, against the oracle (C3 and
  C4 on samples the oracle finishes in seconds).
"""
import math

import numpy as np
import pytest

import paper_1808_01478_gb300 as dh
import workloads as w
from tests.test_autotune_gpu import tune_key, write_cache

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def assert_same(got, want, name=""):
    assert got.shape == want.shape, (got.shape, want.shape)
    if not np.array_equal(got, want):
        bad = np.argwhere(got != want)
        h, k = bad[0]
        raise AssertionError(f"{name}: {len(bad)} bins differ; first (h={h}, bin={k}): "
                             f"gpu {got[h, k]} oracle {want[h, k]}")


def edge_lattices():
    """Integer lattices (13^3 = 2,197 particles: spatially sorted, ragged tiles)
    with dyadic bin widths, so that axis-aligned pairs and Pythagorean pairs sit
    exactly on binary64 thresholds."""
    from tests.test_exactness_pins import edge_lattice_cases

    return edge_lattice_cases()


CASES = edge_lattices()


@pytest.mark.parametrize("coords", ["f32", "f64"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_binary64_replay_runs_and_matches_oracle(torch_mod, oracle_mod, name, coords):
    f = CASES[name]
    x = f.coords.astype(np.float64) if coords == "f64" else f.coords
    want = oracle_mod.histogram(x, f.offsets, f.box_type, f.box, f.r_max, f.nbins)
    with dh.Context(0) as ctx:
        got = ctx.histogram(torch_mod.from_numpy(x).cuda(), f.offsets, f.box_type, f.box, f.r_max, f.nbins)
        st = ctx.stats()
    assert_same(got.cpu().numpy().view(np.uint64), want, f"{name}/{coords}")
    assert st["deferred"] > 0, st
    assert st["exact_fallback"] > 0, st


@pytest.mark.parametrize("name", sorted(CASES))
def test_binary64_replay_in_the_batched_path(torch_mod, oracle_mod, name):
    # the same frames through one persistent launch per variant (CUDA graph)
    f = CASES[name]
    g = w.uniform_frame(71, 3000, f.box_type, f.box if f.box_type != w.BOX_NONE else w.ortho_box(12.0),
                        f.r_max, f.nbins)
    if f.box_type == w.BOX_NONE:
        g = w.frame_from(g.coords, g.offsets, w.BOX_NONE, np.zeros(9), f.r_max, f.nbins, "uniform-none")
    frames = [f, g]
    with dh.Context(0) as ctx:
        fas = [dh.FrameArgs(torch_mod.from_numpy(h.coords).cuda(), h.offsets, h.box_type, h.box, h.r_max, h.nbins)
               for h in frames]
        ctx.histogram_batch(fas)
        st = ctx.stats()
        assert st["graph_replays"] == 1 and st["exact_fallback"] > 0, st
        for fa, h in zip(fas, frames):
            assert_same(fa.out.cpu().numpy().view(np.uint64), oracle_mod.histogram_frame(h), h.name)


def test_uint32_private_counts_flush_before_overflow(torch_mod, oracle_mod, tmp_path):
    # One 256-thread block per SM and a no-box frame of N = 2,000,000 with two
    # bins: each block evaluates about 1.3e10 pairs, about 70 % of them in bin 0,
    # so a block's uint32 count of bin 0 passes 2^32 twice unless it is flushed.
    n, na = 2_000_000, 2048
    rng = w.rng_for(72)
    x = (rng.random((n, 3)) * 100.0).astype(np.float32)
    r_max = 100.0 * math.sqrt(3.0) * 1.0001
    f = w.frame_from(x, [0, na, n], w.BOX_NONE, np.zeros(9), r_max, 2, "flush")
    sms = torch_mod.cuda.get_device_properties(0).multi_processor_count
    path = tmp_path / "tune.txt"
    write_cache(path, sms, [tune_key([f])], 1024, 1, 1, 256)
    with dh.Context(0, tune_cache=str(path)) as ctx:
        out = ctx.histogram(torch_mod.from_numpy(x).cuda(), f.offsets, f.box_type, f.box, f.r_max, f.nbins)
        st = ctx.stats()
    got = out.cpu().numpy().view(np.uint64)
    assert st["blocks_per_sm"] == 1 and st["blocks"] == sms, st
    per_block_bin0 = int(got[2, 0]) / sms
    assert per_block_bin0 > 2 ** 32, per_block_bin0  # the flush must have fired in every block
    assert int(got.sum()) == n * (n - 1) // 2  # every pair in range, counted once
    nb = n - na
    assert int(got[2].sum()) == nb * (nb - 1) // 2
    for k, (a, c) in enumerate([(0, 0), (0, 1)]):
        want = oracle_mod.histogram_one(f.coords, f.offsets, f.box_type, f.box, f.r_max, f.nbins, a, c)
        assert np.array_equal(got[k], want), ((a, c), got[k], want)


def test_c2_full_size(torch_mod, oracle_mod):
    # orthorhombic 60^3, N = 100,000, two species of 50,000, r_max 30, 10,000 bins:
    # all three histograms (5e9 pairs) against the oracle
    f = w.config_ortho_two_species(seed=2)
    with dh.Context(0) as ctx:
        got = ctx.histogram(torch_mod.from_numpy(f.coords).cuda(), f.offsets, f.box_type, f.box, f.r_max,
                            f.nbins).cpu().numpy().view(np.uint64)
        st = ctx.stats()
    assert st["pairs"] == f.n_pairs() and st["deferred"] > 0
    assert_same(got, oracle_mod.histogram_frame(f), "C2")


def test_c3_full_size_sampled(torch_mod, oracle_mod):
    # triclinic 80 A cell (70/80/100 deg), N = 500,000 as 200 Gaussian clusters
    # (sigma 2) plus 20 % background, 3 species, r_max 35, 20,000 bins: the
    # clustered contention case.  The GPU runs the frame as given (6 histograms)
    # and with the first 2,048 particles of species 0 (random in the cell: the
    # generator permutes before labelling) carved out as a species of their own
    # (10 histograms).  The carved species' 4 histograms (1e9 pairs against
    # every particle) are compared with the oracle; the 3-species histograms
    # must equal the sums of the 4-species ones that make them up.
    f = w.config_triclinic_clusters(seed=3)
    o = [int(v) for v in f.offsets]
    na = 2048
    g = w.frame_from(f.coords, [0, na] + o[1:], f.box_type, f.box, f.r_max, f.nbins, "C3-carved")
    with dh.Context(0) as ctx:
        x = torch_mod.from_numpy(f.coords).cuda()
        h3 = ctx.histogram(x, f.offsets, f.box_type, f.box, f.r_max, f.nbins).cpu().numpy().view(np.uint64)
        h4 = ctx.histogram(x, g.offsets, g.box_type, g.box, g.r_max, g.nbins).cpu().numpy().view(np.uint64)
    assert h3.shape == (6, f.nbins) and h4.shape == (10, f.nbins)

    def h(S, a, b):
        return a * S - a * (a - 1) // 2 + (b - a)

    for c in range(4):
        want = oracle_mod.histogram_one(g.coords, g.offsets, g.box_type, g.box, g.r_max, g.nbins, 0, c)
        diff = np.flatnonzero(h4[h(4, 0, c)] != want)
        assert diff.size == 0, ((0, c), diff[:10])
    # species 0 of the frame = carved species 0 + rest 1; species 1, 2 -> 2, 3
    m = {0: [0, 1], 1: [2], 2: [3]}
    for a in range(3):
        for b in range(a, 3):
            s = np.zeros(f.nbins, np.uint64)
            for p in m[a]:
                for q in m[b]:
                    if a == b and q < p:
                        continue
                    s += h4[h(4, min(p, q), max(p, q))]
            assert np.array_equal(h3[h(3, a, b)], s), (a, b)


def test_c4_batch_sampled_against_oracle(torch_mod, oracle_mod):
    # the 256-frame batch the bench times (orthorhombic, N log-uniform in
    # [5,000, 200,000], 30/70 species, r_max L/2, 4,096 bins), one batched call
    # replayed as a CUDA graph; every frame with N <= 11,700 (58 frames) and
    # four others drawn at random up to N = 60,000 against the oracle
    frames = w.batch_frames(seed=7, n_frames=256)
    with dh.Context(0) as ctx:
        fas = [dh.FrameArgs(torch_mod.from_numpy(f.coords).cuda(), f.offsets, f.box_type, f.box, f.r_max, f.nbins)
               for f in frames]
        ctx.histogram_batch(fas)
        assert ctx.stats()["graph_replays"] == 1
        got = [fa.out.cpu().numpy().view(np.uint64) for fa in fas]
    small = [k for k, f in enumerate(frames) if f.n <= 11_700]
    rest = [k for k, f in enumerate(frames) if 11_700 < f.n <= 60_000]
    pick = small + sorted(w.rng_for(73).choice(rest, size=4, replace=False).tolist())
    assert len(small) >= 50
    for k in pick:
        assert_same(got[k], oracle_mod.histogram_frame(frames[k]), frames[k].name)
