"""Trajectory accumulation and g(r) on the device (dh_rdf, Eq. 1).

Frames of a trajectory are summed into one histogram with DH_ACCUMULATE (an
integer sum: bit-exact against the oracle's per-frame histograms added up),
then dh_rdf normalises it.  g is binary64 on both sides; the GPU evaluates the
shell volume as (4 pi / 3) dr^3 (3k(k+1) + 1) while the oracle subtracts the
two cubes, whose cancellation costs up to about k ulps, so the tolerance is
relative 4e-16 x (nbins + 16) (plus the few roundings of the quotient).
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


def pair_densities(f, volume):
    sizes = f.species_sizes()
    dens = []
    for a in range(len(sizes)):
        for b in range(a, len(sizes)):
            p = sizes[a] * (sizes[a] - 1) / 2 if a == b else sizes[a] * sizes[b]
            dens.append(p / volume)
    return dens


def test_rdf_of_an_accumulated_trajectory(torch_mod, oracle_mod):
    box = w.ortho_box(30.0, 26.0, 34.0)
    r_max, nbins = 12.5, 2500
    frames = [w.uniform_frame(40 + k, 5000, w.BOX_ORTHO, box, r_max, nbins, n_species=2) for k in range(3)]
    dens = pair_densities(frames[0], w.box_volume(box))
    with dh.Context(0) as ctx:
        acc = torch_mod.zeros((3, nbins), dtype=torch_mod.int64, device="cuda")
        for f in frames:
            ctx.histogram(torch_mod.from_numpy(f.coords).cuda(), f.offsets, f.box_type, f.box, f.r_max, f.nbins,
                          acc, accumulate=True)
        total = sum(oracle_mod.histogram_frame(f) for f in frames)
        assert np.array_equal(acc.cpu().numpy().view(np.uint64), total)
        g = ctx.rdf(acc, r_max, dens, len(frames)).cpu().numpy()
    want = oracle_mod.rdf(total, r_max, dens, len(frames))
    np.testing.assert_allclose(g, want, rtol=4e-16 * (nbins + 16), atol=0)
    # an ideal gas: g is 1 up to counting noise (mean weighted by the shell volumes)
    k = np.arange(nbins, dtype=np.float64)
    for h in range(3):
        assert abs(np.average(g[h], weights=3 * k * (k + 1) + 1) - 1.0) < 0.01


def test_rdf_hand_shells_on_device(torch_mod, oracle_mod):
    counts = torch_mod.tensor([[1, 7, 19], [2, 14, 38]], dtype=torch_mod.int64, device="cuda")
    dens = [3.0 / (4.0 * math.pi), 3.0 / (2.0 * math.pi)]
    with dh.Context(0) as ctx:
        g = ctx.rdf(counts, 3.0, dens, 1).cpu().numpy()
    np.testing.assert_allclose(g, np.ones((2, 3)), rtol=4e-15, atol=0)
    np.testing.assert_allclose(g, oracle_mod.rdf(counts.cpu().numpy().astype(np.uint64), 3.0, dens, 1),
                               rtol=4e-15, atol=0)


def test_rdf_wide_histogram(torch_mod, oracle_mod):
    # a multi-sweep histogram's g: the largest k of the tolerance argument
    nbins = 150_000
    rng = np.random.default_rng(3)
    c = rng.integers(0, 1000, size=(1, nbins)).astype(np.int64)
    with dh.Context(0) as ctx:
        g = ctx.rdf(torch_mod.from_numpy(c).cuda(), 40.0, [0.7], 5).cpu().numpy()
    np.testing.assert_allclose(g, oracle_mod.rdf(c.astype(np.uint64), 40.0, [0.7], 5),
                               rtol=4e-16 * (nbins + 16), atol=0)


def test_rdf_rejects_bad_arguments(torch_mod):
    counts = torch_mod.zeros((1, 10), dtype=torch_mod.int64, device="cuda")
    with dh.Context(0) as ctx:
        for r_max, dens, frames in [(0.0, [1.0], 1), (5.0, [0.0], 1), (5.0, [1.0], 0), (float("inf"), [1.0], 1)]:
            with pytest.raises(dh.DHError) as e:
                ctx.rdf(counts, r_max, dens, frames)
            assert e.value.status == dh.DH_ERR_INVALID
