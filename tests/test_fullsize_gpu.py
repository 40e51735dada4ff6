"""Parity at the full size of the headline workload: N = 1,000,000 per frame.

The oracle cannot evaluate the 5e11 pairs of a headline frame inside a test, so
each frame is split into a sampled species A, its first 2,048 particles (the
generator is uniform, so they are a random subset of the box), and B, the rest.
The three frames (no box, orthorhombic, triclinic) go through one batched call,
the launch configuration the bench times: one persistent launch per variant,
replayed as a CUDA graph, with the spatial order and the tile images of the
full-size frames.  The AA and AB histograms (2e9 pairs per frame, against every
particle of the box) are compared with the oracle bin for bin; BB is checked by
the pair-count invariant where it holds (no box: every pair is in range).
"""
import numpy as np
import pytest

import paper_1808_01478_gb300 as dh
import workloads as w

pytestmark = pytest.mark.gpu

N = 1_000_000
NA = 2048


@pytest.fixture(scope="module")
def torch_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def split_frame(box_type, seed):
    f = w.headline_frame(box_type, seed=seed, n=N)
    return w.frame_from(f.coords, [0, NA, N], f.box_type, f.box, f.r_max, f.nbins, f.name + "-split")


def test_headline_frames_at_full_size(torch_mod, oracle_mod):
    frames = [split_frame(b, 11 + b) for b in (w.BOX_NONE, w.BOX_ORTHO, w.BOX_TRICLINIC)]
    with dh.Context(0) as ctx:
        fas = [dh.FrameArgs(torch_mod.from_numpy(f.coords).cuda(), f.offsets, f.box_type, f.box, f.r_max, f.nbins)
               for f in frames]
        ctx.histogram_batch(fas)
        st = ctx.stats()
        got = [fa.out.cpu().numpy().view(np.uint64) for fa in fas]
    assert st["uniform_pairs"] > 0 and st["axis_pairs"] > 0, st
    for f, g in zip(frames, got):
        assert g.shape == (3, f.nbins)
        for k, (a, c) in enumerate([(0, 0), (0, 1)]):
            want = oracle_mod.histogram_one(f.coords, f.offsets, f.box_type, f.box, f.r_max, f.nbins, a, c)
            diff = np.flatnonzero(g[k] != want)
            assert diff.size == 0, (f.name, (a, c), diff[:10], g[k][diff[:10]], want[diff[:10]])
        if f.box_type == w.BOX_NONE:  # r_max is the cube's diagonal: every pair counted once
            nb = N - NA
            assert int(g[2].sum()) == nb * (nb - 1) // 2
            assert int(g.sum()) == N * (N - 1) // 2
