"""Binary64 input coordinates (DH_COORDS_F64) against the binary64-input oracle.

The coordinates use all 53 bits, so the distance vector of the definition is
rounded once per component; the GPU decides most pairs from the coordinates
rounded to float32 (the error bound includes that rounding) and re-decides the
rest from the binary64 values.  Counts are integers: bit-exact on every bin.
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
    c = dh.Context(0)
    yield c
    c.close()


def f64_frame(seed, n, box_type, box, r_max, nbins, n_species=1, extent=None):
    """Uniform particles with binary64 coordinates (not float32 values)."""
    rng = w.rng_for(seed)
    if box_type == w.BOX_TRICLINIC:
        x = (w.box_matrix(box) @ rng.random((n, 3)).T).T
    else:
        L = np.asarray(extent if extent is not None else [box[0], box[4], box[8]], dtype=np.float64)
        x = rng.random((n, 3)) * L
    return np.ascontiguousarray(x, dtype=np.float64), w.even_offsets(n, n_species)


TRIC = w.triclinic_box(30, 30, 30, *w.C3_ANGLES)
CASES = {
    "nobox": (41, 3100, w.BOX_NONE, None, 9.0, 1500, 1, [7.0, 6.0, 8.0]),
    "ortho_2species": (42, 5000, w.BOX_ORTHO, w.ortho_box(20.0, 24.0, 17.0), 8.5, 4000, 2, None),
    "tric": (43, 4000, w.BOX_TRICLINIC, TRIC, 0.95 * float(w.box_heights(TRIC).min()) / 2, 3000, 1, None),
    "tric_search": (44, 2500, w.BOX_TRICLINIC, TRIC, 20.0, 2500, 2, None),
    "ortho_sorted": (45, 9000, w.BOX_ORTHO, w.ortho_box(30.0), 15.0, 6000, 1, None),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("where", ["device", "host"])
def test_f64_parity(ctx, torch_mod, oracle_mod, name, where):
    seed, n, bt, box, r_max, nbins, ns, ext = CASES[name]
    x, offs = f64_frame(seed, n, bt, box, r_max, nbins, ns, ext)
    want = oracle_mod.histogram(x, offs, bt, box, r_max, nbins)
    if where == "device":
        got = ctx.histogram(torch_mod.from_numpy(x).cuda(), offs, bt, box, r_max, nbins)
        got = got.cpu().numpy().view(np.uint64)
    else:
        got = ctx.histogram(x, offs, bt, box, r_max, nbins)
    assert np.array_equal(got, want), (name, int((got != want).sum()))


def test_f64_on_bin_edges(ctx, torch_mod, oracle_mod):
    # a lattice whose spacing is the bin width, in binary64: many pairs lie on or
    # within a few ulps of an edge
    g = np.arange(14, dtype=np.float64) * 0.1 + 0.05
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    x = x + np.float64(1e-12) * w.rng_for(46).standard_normal(x.shape)
    box = w.ortho_box(1.4)
    want = oracle_mod.histogram(x, [0, len(x)], w.BOX_ORTHO, box, 0.7, 7)
    got = ctx.histogram(torch_mod.from_numpy(np.ascontiguousarray(x)).cuda(), [0, len(x)], w.BOX_ORTHO, box, 0.7, 7)
    assert np.array_equal(got.cpu().numpy().view(np.uint64), want)


def test_f64_in_a_mixed_batch(torch_mod, oracle_mod):
    frames = []
    for name in ("ortho_2species", "tric", "nobox"):
        seed, n, bt, box, r_max, nbins, ns, ext = CASES[name]
        x, offs = f64_frame(seed + 100, n, bt, box, r_max, nbins, ns, ext)
        frames.append((x, offs, bt, box, r_max, nbins))
    f32 = w.uniform_frame(47, 3000, w.BOX_ORTHO, w.ortho_box(15.0), 7.0, 2000)
    with dh.Context(0) as ctx:
        fas = [dh.FrameArgs(torch_mod.from_numpy(x).cuda(), o, bt, b, r, k) for x, o, bt, b, r, k in frames]
        fas.append(dh.FrameArgs(torch_mod.from_numpy(f32.coords).cuda(), f32.offsets, f32.box_type, f32.box,
                                f32.r_max, f32.nbins))
        ctx.histogram_batch(fas)
        for fa, (x, o, bt, b, r, k) in zip(fas, frames):
            assert np.array_equal(fa.out.cpu().numpy().view(np.uint64), oracle_mod.histogram(x, o, bt, b, r, k))
        assert np.array_equal(fas[-1].out.cpu().numpy().view(np.uint64), oracle_mod.histogram_frame(f32))


def test_f64_rejected_where_not_supported(torch_mod):
    x, offs = f64_frame(48, 500, w.BOX_ORTHO, w.ortho_box(10.0), 5.0, 100)
    xd = torch_mod.from_numpy(x).cuda()
    fa = dh.FrameArgs(xd, offs, w.BOX_ORTHO, w.ortho_box(10.0), 5.0, 100)
    with pytest.raises(dh.DHError) as e:
        dh.dh_histogram_noalloc(fa.frame)
    assert e.value.status == dh.DH_ERR_INVALID
    with dh.Context(0) as ctx:
        with pytest.raises(dh.DHError) as e:
            ctx.submit(fa)
        assert e.value.status == dh.DH_ERR_INVALID
