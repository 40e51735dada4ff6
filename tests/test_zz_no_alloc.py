"""dh_histogram_noalloc: the allocation-free entry point.

Callers that may not allocate device memory (code under a framework's own
caching allocator, which a cudaMalloc behind its back would fragment or
overcommit; processes with a fixed device-memory budget) use this variant: it
keeps its scratch in a fixed device array inside the library.  Its output must
equal the regular dh_histogram bin for bin (the integer tolerance of every
parity test here), call after call, since all calls share that array, and the
FP64 oracle as well.

This file is named so pytest collects it last; it also passes on its own in a
fresh process.
"""
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
    torch.cuda.set_device(0)
    return torch


def noalloc(torch, f, x, stream=None):
    out = torch.zeros((f.n_hist, f.nbins), dtype=torch.int64, device=x.device)
    fa = dh.FrameArgs(x, f.offsets, f.box_type, f.box, f.r_max, f.nbins, out)
    dh.dh_histogram_noalloc(fa.frame, None if stream is None else stream.cuda_stream)
    return out.cpu().numpy().view(np.uint64).copy()


FRAMES = [
    w.uniform_frame(21, 60000, w.BOX_ORTHO, w.ortho_box(60.0), 30.0, 4096, n_species=2),
    w.config_triclinic_clusters(seed=22, n=40000, n_clusters=30, edge=80.0, nbins=20000),
    w.uniform_frame(23, 9000, w.BOX_NONE, w.ortho_box(20.0), 35.0, 60000),
]


@pytest.fixture(scope="module")
def oracle_lib():
    import oracle

    oracle.build()
    return oracle


@pytest.mark.parametrize("k", range(len(FRAMES)))
def test_noalloc_matches_dh_histogram_on_two_calls(torch_mod, oracle_lib, k):
    f = FRAMES[k]
    x = torch_mod.from_numpy(f.coords).cuda()
    with dh.Context(0) as ctx:
        ref = ctx.histogram(x, f.offsets, f.box_type, f.box, f.r_max, f.nbins).cpu().numpy().view(np.uint64)
    first = noalloc(torch_mod, f, x)
    second = noalloc(torch_mod, f, x)
    assert np.array_equal(first, ref), f.name
    assert np.array_equal(second, ref), f.name
    assert np.array_equal(first, oracle_lib.histogram_frame(f)), f.name


def test_noalloc_on_a_stream_and_after_another_frame(torch_mod):
    s = torch_mod.cuda.Stream()
    a, b = FRAMES[1], FRAMES[0]
    xa = torch_mod.from_numpy(a.coords).cuda()
    xb = torch_mod.from_numpy(b.coords).cuda()
    with dh.Context(0) as ctx:
        ref_b = ctx.histogram(xb, b.offsets, b.box_type, b.box, b.r_max, b.nbins).cpu().numpy().view(np.uint64)
    noalloc(torch_mod, a, xa, s)
    got_b = noalloc(torch_mod, b, xb, s)
    assert np.array_equal(got_b, ref_b)


def test_noalloc_rejects_frames_beyond_its_limits(torch_mod):
    f = w.uniform_frame(24, dh.DH_NOALLOC_MAX_N + 1, w.BOX_NONE, w.ortho_box(10.0), 5.0, 16)
    x = torch_mod.from_numpy(f.coords).cuda()
    out = torch_mod.zeros((1, 16), dtype=torch_mod.int64, device=x.device)
    fa = dh.FrameArgs(x, f.offsets, f.box_type, f.box, f.r_max, f.nbins, out)
    with pytest.raises(dh.DHError) as e:
        dh.dh_histogram_noalloc(fa.frame)
    assert e.value.status == dh.DH_ERR_INVALID
    g = FRAMES[0]
    xg = torch_mod.from_numpy(g.coords).cuda()
    out = torch_mod.zeros((g.n_hist, dh.DH_NOALLOC_MAX_BINS + 1), dtype=torch_mod.int64, device=x.device)
    fa = dh.FrameArgs(xg, g.offsets, g.box_type, g.box, g.r_max, dh.DH_NOALLOC_MAX_BINS + 1, out)
    with pytest.raises(dh.DHError) as e:
        dh.dh_histogram_noalloc(fa.frame)
    assert e.value.status == dh.DH_ERR_INVALID
    fh = dh.FrameArgs(g.coords, g.offsets, g.box_type, g.box, g.r_max, g.nbins)  # host pointers
    with pytest.raises(dh.DHError) as e:
        dh.dh_histogram_noalloc(fh.frame)
    assert e.value.status == dh.DH_ERR_INVALID
    # more species pairs than work segments: rejected before any work, out untouched
    n = 1000
    many = w.uniform_frame(25, n, w.BOX_NONE, w.ortho_box(10.0), 5.0, 64, n_species=40)
    xm = torch_mod.from_numpy(many.coords).cuda()
    out = torch_mod.full((many.n_hist, 64), 7, dtype=torch_mod.int64, device=xm.device)
    fa = dh.FrameArgs(xm, many.offsets, many.box_type, many.box, many.r_max, many.nbins, out)
    with pytest.raises(dh.DHError) as e:
        dh.dh_histogram_noalloc(fa.frame)
    assert e.value.status == dh.DH_ERR_INVALID
    assert bool((out == 7).all())
