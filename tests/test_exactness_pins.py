"""CPU pins of the edge lattices used by the exactness tests on the GPU.

The GPU's binary64 replay only runs for pairs whose r^2 the double-float tier
cannot separate from a bin threshold T[k] (the smallest binary64 r^2 whose bin
of Alg. 1 is >= k).  These fixtures are meant to hold such pairs; this file
checks, with the oracle alone, that they do: many pairs have r^2 exactly equal
to T[k] (the oracle's bin of r^2 is k, of the binary64 value just below it
k - 1), and each frame is of the minimum-image variant it stands for.
"""
import math

import numpy as np
import pytest

import workloads as w

P = 13  # particles per lattice side: 2,197 particles


def _lattice():
    g = np.arange(P, dtype=np.float64)
    return np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).astype(np.float32)


TRIC_BOX = np.array([13.0, 3.0, 2.0, 0.0, 13.0, 3.0, 0.0, 0.0, 13.0])


def edge_lattice_cases():
    x = _lattice()
    n = x.shape[0]
    return {
        # dr = 1, r_max beyond the diagonal 12 sqrt(3): every pair counted
        "none": w.frame_from(x, [0, n], w.BOX_NONE, np.zeros(9), 24.0, 24, "edge-none"),
        # the lattice fills the periodic cube; dr = 0.5; two species
        "ortho": w.frame_from(x, [0, 1000, n], w.BOX_ORTHO, w.ortho_box(13.0), 6.5, 13, "edge-ortho"),
        # triclinic, r_max below half the smallest plane spacing (one wrap, m = 0 shortcut)
        "tric": w.frame_from(x, [0, n], w.BOX_TRICLINIC, TRIC_BOX, 6.0, 12, "edge-tric"),
        # the same cell with r_max beyond it: Eq. 5 wrap plus the 27-image search
        "tric_search": w.frame_from(x, [0, 700, n], w.BOX_TRICLINIC, TRIC_BOX, 10.0, 20, "edge-tric-search"),
    }


def test_edge_lattice_variants():
    cases = edge_lattice_cases()
    h_min = float(w.box_heights(TRIC_BOX).min())
    assert cases["tric"].r_max <= (1.0 - 2.0 ** -8) * h_min / 2.0
    assert cases["tric_search"].r_max > h_min / 2.0
    # reduced triclinic form: |bx|, |cx| <= ax/2 and |cy| <= by/2
    assert abs(TRIC_BOX[1]) <= TRIC_BOX[0] / 2 and abs(TRIC_BOX[2]) <= TRIC_BOX[0] / 2
    assert abs(TRIC_BOX[5]) <= TRIC_BOX[4] / 2
    f = cases["none"]
    assert f.r_max > 12.0 * math.sqrt(3.0)


@pytest.mark.parametrize("name", sorted(edge_lattice_cases()))
def test_edge_lattices_put_pairs_on_binary64_thresholds(oracle_mod, name):
    f = edge_lattice_cases()[name]
    rng = w.rng_for(5)
    n = f.coords.shape[0]
    ii = rng.integers(0, n, size=20000)
    jj = rng.integers(0, n, size=20000)
    keep = ii != jj
    r2 = oracle_mod.pairs_r2(f.coords, ii[keep], jj[keep], f.box_type, f.box)
    on_edge = 0
    for q in r2:
        k = oracle_mod.bin_of(q, f.r_max, f.nbins)
        if 1 <= k < f.nbins and oracle_mod.bin_of(float(np.nextafter(q, 0.0)), f.r_max, f.nbins) == k - 1:
            on_edge += 1
    # a few percent of random pairs lie exactly on an edge (axis-aligned and
    # Pythagorean displacements whose length is a multiple of the bin width)
    assert on_edge >= 100, on_edge
