"""Served path (dh_submit / dh_poll / dh_wait / dh_cancel): continuous batching.

Each request's result must equal the FP64 oracle and be identical whether the
request runs alone or mixed with others that arrive while it is on the GPU.
Failures are injected on the host only (cancel, tiny timeouts, an exhausted
pool, invalid frames).
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
    return torch


@pytest.fixture(scope="module")
def ctx(torch_mod):
    c = dh.Context(0, pool_bytes=1 << 30, max_inflight=16)
    yield c
    c.close()


def mixed_frames(seed=0, k=10, n_lo=500, n_hi=6000):
    rng = w.rng_for(seed)
    return [w.served_request(rng, n_lo=n_lo, n_hi=n_hi) for _ in range(k)]


def submit(ctx, f):
    fa = dh.FrameArgs(f.coords, f.offsets, f.box_type, f.box, f.r_max, f.nbins)
    return ctx.submit(fa), fa


def test_served_results_match_oracle(ctx, oracle_mod):
    frames = mixed_frames(1)
    subs = [submit(ctx, f) for f in frames]
    for (t, fa), f in zip(subs, frames):
        assert ctx.wait(t) == dh.DH_OK
        want = oracle_mod.histogram_frame(f)
        assert np.array_equal(fa.out, want), f.name
    # a final status is reported once
    assert ctx.poll(subs[0][0]) == dh.DH_ERR_NOTFOUND


def test_alone_equals_mixed(ctx, oracle_mod):
    probe = w.uniform_frame(3, 5000, w.BOX_TRICLINIC, w.triclinic_box(40, 40, 40, *w.C3_ANGLES), 17.0, 4096,
                            n_species=2)
    t, fa = submit(ctx, probe)
    assert ctx.wait(t) == dh.DH_OK
    alone = fa.out.copy()
    # large requests first, then the probe in the middle of the stream
    big = [w.uniform_frame(10 + k, 60000, w.BOX_ORTHO, w.ortho_box(80.0), 40.0, 8192, n_species=3)
           for k in range(2)]
    subs = [submit(ctx, f) for f in big]
    subs += [submit(ctx, f) for f in mixed_frames(2, k=6)]
    tp, fap = submit(ctx, probe)
    subs += [submit(ctx, f) for f in mixed_frames(3, k=6)]
    assert ctx.wait(tp) == dh.DH_OK
    for t, _ in subs:
        assert ctx.wait(t) == dh.DH_OK
    assert np.array_equal(alone, fap.out)
    assert np.array_equal(alone, oracle_mod.histogram_frame(probe))
    # and the large ones are right as well (checked by the pair-count invariant)
    for (t, fa), f in zip(subs[:2], big):
        assert int(fa.out.sum()) > 0
        assert int(fa.out[1].sum()) <= f.species_sizes()[0] * f.species_sizes()[1]


def test_served_device_pointers(ctx, torch_mod, oracle_mod):
    f = w.uniform_frame(5, 7000, w.BOX_ORTHO, w.ortho_box(30.0), 15.0, 3000, n_species=2)
    x = torch_mod.from_numpy(f.coords).cuda()
    fa = dh.FrameArgs(x, f.offsets, f.box_type, f.box, f.r_max, f.nbins)
    t = ctx.submit(fa)
    assert ctx.wait(t) == dh.DH_OK
    got = fa.out.cpu().numpy().view(np.uint64)
    assert np.array_equal(got, oracle_mod.histogram_frame(f))


def test_cancel_and_timeout(ctx):
    big = w.uniform_frame(7, 400_000, w.BOX_TRICLINIC, w.scale_box(w.triclinic_box(1, 1, 1, *w.C3_ANGLES), 4e6),
                          60.0, 16384)
    t, fa = submit(ctx, big)
    assert ctx.wait(t, timeout_ns=1_000) == dh.DH_ERR_TIMEOUT
    assert ctx.poll(t) == dh.DH_PENDING
    assert ctx.cancel(t) == dh.DH_OK
    st = ctx.wait(t)
    assert st in (dh.DH_ERR_CANCELLED, dh.DH_OK)
    # the server keeps serving
    f = mixed_frames(4, k=1)[0]
    t2, _ = submit(ctx, f)
    assert ctx.wait(t2) == dh.DH_OK


def test_unknown_ticket_and_invalid_frame(ctx):
    assert ctx.poll(987654321) == dh.DH_ERR_NOTFOUND
    assert ctx.wait(987654321, 1000) == dh.DH_ERR_NOTFOUND
    x = np.zeros((4, 3), np.float32)
    fa = dh.FrameArgs(x, [0, 4], w.BOX_NONE, None, -1.0, 8)
    with pytest.raises(dh.DHError) as e:
        ctx.submit(fa)
    assert e.value.status == dh.DH_ERR_INVALID
    x[1, 1] = np.inf
    fa = dh.FrameArgs(x, [0, 4], w.BOX_NONE, None, 1.0, 8)
    t = ctx.submit(fa)
    assert ctx.wait(t) == dh.DH_ERR_INVALID


def test_admission_by_footprint(torch_mod, oracle_mod):
    # a pool that holds only a few requests at a time: the rest queue and still finish
    with dh.Context(0, pool_bytes=3 << 20, max_inflight=4) as c:
        frames = mixed_frames(6, k=12, n_lo=2000, n_hi=20000)
        subs = [submit(c, f) for f in frames]
        for (t, fa), f in zip(subs, frames):
            assert c.wait(t) == dh.DH_OK
            assert np.array_equal(fa.out, oracle_mod.histogram_frame(f))
        huge = w.uniform_frame(1, 300_000, w.BOX_NONE, w.ortho_box(10.0), 20.0, 100)
        with pytest.raises(dh.DHError) as e:
            submit(c, huge)
        assert e.value.status == dh.DH_ERR_NOMEM


def test_request_deadline(torch_mod, oracle_mod):
    # dh_config.timeout_ns: a request not finished that long after dh_submit is
    # cancelled and reports DH_ERR_TIMEOUT, queued or running; requests that
    # finish in time are unaffected and the server keeps serving
    big = w.uniform_frame(8, 600_000, w.BOX_TRICLINIC, w.scale_box(w.triclinic_box(1, 1, 1, *w.C3_ANGLES), 6e6),
                          60.0, 16384)
    with dh.Context(0, pool_bytes=1 << 30, max_inflight=4, timeout_ns=20_000_000) as c:
        t_big, _ = submit(c, big)
        assert c.wait(t_big, timeout_ns=30_000_000_000) == dh.DH_ERR_TIMEOUT
        f = mixed_frames(9, k=1, n_lo=800, n_hi=1500)[0]
        t, fa = submit(c, f)
        assert c.wait(t) == dh.DH_OK
        assert np.array_equal(fa.out, oracle_mod.histogram_frame(f))
