"""Batched path (dh_histogram_batch): many frames of uneven N, species, box and
bin counts through one launch per minimum-image variant, replayed as a CUDA
graph for device pointers.  Every frame must equal the FP64 oracle, and the
batch must equal the per-frame plain path bit for bit."""
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


def mixed_batch(seed=0):
    rng = w.rng_for(seed)
    frames = [w.served_request(rng, n_lo=300, n_hi=5000) for _ in range(10)]
    frames.append(w.uniform_frame(seed + 1, 2000, w.BOX_ORTHO, w.ortho_box(30.0), 15.0, 70_000, n_species=2))
    frames.append(w.uniform_frame(seed + 2, 1500, w.BOX_TRICLINIC, w.triclinic_box(20, 20, 20, *w.C3_ANGLES),
                                  14.0, 900))  # r_max beyond half the plane spacing: 27-image search
    frames.append(w.frame_from(np.zeros((0, 3), np.float32), [0, 0], w.BOX_NONE, np.zeros(9), 1.0, 8, "empty"))
    return frames


def device_args(torch, frames):
    return [dh.FrameArgs(torch.from_numpy(f.coords).cuda(), f.offsets, f.box_type, f.box, f.r_max, f.nbins)
            for f in frames]


def result(torch, fa):
    o = fa.out
    return o.cpu().numpy().view(np.uint64) if hasattr(o, "is_cuda") else o


@pytest.mark.parametrize("cfg_flags", [0, dh.DH_CFG_NO_GRAPH])
def test_batch_matches_oracle_and_plain(torch_mod, oracle_mod, cfg_flags):
    frames = mixed_batch(3)
    with dh.Context(0, flags=cfg_flags) as ctx:
        fas = device_args(torch_mod, frames)
        ctx.histogram_batch(fas)
        st = ctx.stats()
        assert st["graph_replays"] == (0 if cfg_flags else 1)
        assert st["sweeps"] >= 2
        for fa, f in zip(fas, frames):
            assert np.array_equal(result(torch_mod, fa), oracle_mod.histogram_frame(f)), f.name
        # replay with new inputs of the same shape: graph update path
        fas2 = device_args(torch_mod, frames)
        ctx.histogram_batch(fas2)
        for fa, fb in zip(fas, fas2):
            assert np.array_equal(result(torch_mod, fa), result(torch_mod, fb))
        # per-frame plain path
        for fa, f in zip(fas, frames):
            x = torch_mod.from_numpy(f.coords).cuda()
            got = ctx.histogram(x, f.offsets, f.box_type, f.box, f.r_max, f.nbins)
            assert np.array_equal(got.cpu().numpy().view(np.uint64), result(torch_mod, fa)), f.name


def test_batch_host_pointers(torch_mod, oracle_mod):
    frames = mixed_batch(4)
    with dh.Context(0) as ctx:
        fas = [dh.FrameArgs(f.coords, f.offsets, f.box_type, f.box, f.r_max, f.nbins) for f in frames]
        ctx.histogram_batch(fas)
        assert ctx.stats()["graph_replays"] == 0
        for fa, f in zip(fas, frames):
            assert np.array_equal(fa.out, oracle_mod.histogram_frame(f)), f.name


def test_batch_c4_shape(torch_mod, oracle_mod):
    # the batched workload's shape (orthorhombic, 30/70 species, r_max = L/2,
    # 4,096 bins, log-uniform N) at sizes the oracle finishes quickly
    frames = w.batch_frames(seed=5, n_frames=24, n_lo=500, n_hi=6000)
    with dh.Context(0) as ctx:
        fas = device_args(torch_mod, frames)
        ctx.histogram_batch(fas)
        for fa, f in zip(fas, frames):
            assert np.array_equal(result(torch_mod, fa), oracle_mod.histogram_frame(f)), f.name


def test_batch_rejects_mixed_pointer_kinds(torch_mod):
    frames = mixed_batch(6)[:2]
    with dh.Context(0) as ctx:
        fas = [dh.FrameArgs(torch_mod.from_numpy(frames[0].coords).cuda(), frames[0].offsets, frames[0].box_type,
                            frames[0].box, frames[0].r_max, frames[0].nbins),
               dh.FrameArgs(frames[1].coords, frames[1].offsets, frames[1].box_type, frames[1].box,
                            frames[1].r_max, frames[1].nbins)]
        with pytest.raises(dh.DHError) as e:
            ctx.histogram_batch(fas)
        assert e.value.status == dh.DH_ERR_INVALID


def test_batch_graph_with_timing_events(torch_mod, oracle_mod):
    frames = mixed_batch(8)[:6]
    with dh.Context(0, flags=dh.DH_CFG_TIMING) as ctx:
        fas = device_args(torch_mod, frames)
        ctx.histogram_batch(fas)
        st = ctx.stats()
        assert st["graph_replays"] == 1 and st["pair_kernel_ms"] > 0.0
        for fa, f in zip(fas, frames):
            assert np.array_equal(result(torch_mod, fa), oracle_mod.histogram_frame(f)), f.name
