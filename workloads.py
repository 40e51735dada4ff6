"""Seeded synthetic frames for the particle-pair distance histogram.

This module only builds inputs: coordinates, species offsets, box matrices,
``r_max`` and ``nbins``.  It holds none of the histogram arithmetic (no
distances, no minimum image, no binning), so the FP64 oracle and the CUDA path
can both be fed from it without sharing any of the method's code.

Every generator takes an explicit integer seed and draws from
``numpy.random.Generator(PCG64(seed))``.  Coordinates are float32, the
precision the paper benchmarks in (Sec. 4: all runs in single precision,
particles at pseudo-random positions in a box).

Box matrices are 9 float64 values, row-major 3x3, whose COLUMNS are the box
vectors a, b, c (the matrix B of Eq. 5).  Triclinic boxes are upper triangular:
a = (ax,0,0), b = (bx,by,0), c = (cx,cy,cz).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BOX_NONE = 0
BOX_ORTHO = 1
BOX_TRICLINIC = 2
BOX_NAMES = {BOX_NONE: "none", BOX_ORTHO: "ortho", BOX_TRICLINIC: "triclinic"}


@dataclasses.dataclass
class Frame:
    """One trajectory frame: coordinates of all species, packed contiguously."""

    coords: np.ndarray  # (n, 3) float32, species are contiguous segments
    offsets: np.ndarray  # (S+1,) int64, offsets[0]=0, offsets[S]=n
    box_type: int
    box: np.ndarray  # (9,) float64, row-major, columns = box vectors
    r_max: float
    nbins: int
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.coords.shape[0])

    @property
    def n_species(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def n_hist(self) -> int:
        s = self.n_species
        return s * (s + 1) // 2

    def species_sizes(self) -> list[int]:
        return [int(self.offsets[k + 1] - self.offsets[k]) for k in range(self.n_species)]

    def n_pairs(self) -> int:
        """Unique pairs evaluated: N(N-1)/2 per species plus Na*Nb per species pair."""
        sz = self.species_sizes()
        tot = 0
        for a in range(len(sz)):
            tot += sz[a] * (sz[a] - 1) // 2
            for b in range(a + 1, len(sz)):
                tot += sz[a] * sz[b]
        return tot


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ----------------------------------------------------------------- boxes


def ortho_box(lx: float, ly: float | None = None, lz: float | None = None) -> np.ndarray:
    ly = lx if ly is None else ly
    lz = lx if lz is None else lz
    return np.array([lx, 0, 0, 0, ly, 0, 0, 0, lz], dtype=np.float64)


def triclinic_box(a: float, b: float, c: float, alpha: float, beta: float, gamma: float) -> np.ndarray:
    """Upper-triangular box matrix (columns a, b, c) from lengths and angles in degrees.

    a along x, b in the xy plane; the standard crystallographic construction.
    """
    al, be, ga = (math.radians(v) for v in (alpha, beta, gamma))
    ax = a
    bx, by = b * math.cos(ga), b * math.sin(ga)
    cx = c * math.cos(be)
    cy = c * (math.cos(al) - math.cos(be) * math.cos(ga)) / math.sin(ga)
    cz = c * math.sqrt(max(0.0, 1.0 - math.cos(be) ** 2 - (cy / c) ** 2))
    return np.array([ax, bx, cx, 0.0, by, cy, 0.0, 0.0, cz], dtype=np.float64)


def box_matrix(box: np.ndarray) -> np.ndarray:
    return np.asarray(box, dtype=np.float64).reshape(3, 3)


def box_volume(box: np.ndarray) -> float:
    return float(abs(np.linalg.det(box_matrix(box))))


def box_heights(box: np.ndarray) -> np.ndarray:
    """Distances between opposite faces of the cell (plane spacings), one per box vector."""
    m = box_matrix(box)
    a, b, c = m[:, 0], m[:, 1], m[:, 2]
    v = box_volume(box)
    return np.array([v / np.linalg.norm(np.cross(b, c)),
                     v / np.linalg.norm(np.cross(c, a)),
                     v / np.linalg.norm(np.cross(a, b))])


def scale_box(box: np.ndarray, volume: float) -> np.ndarray:
    f = (volume / box_volume(box)) ** (1.0 / 3.0)
    return np.asarray(box, dtype=np.float64) * f


def wrap_into_cell(x: np.ndarray, box: np.ndarray) -> np.ndarray:
    """Map positions (float64) into the primary cell: fractional coordinates in [0,1)."""
    m = box_matrix(box)
    s = np.linalg.solve(m, x.T).T
    s -= np.floor(s)
    return (m @ s.T).T


# ----------------------------------------------------------------- frames


def uniform_in_cell(rng: np.random.Generator, n: int, box: np.ndarray) -> np.ndarray:
    s = rng.random((n, 3))
    return (box_matrix(box) @ s.T).T.astype(np.float32)


def even_offsets(n: int, n_species: int) -> np.ndarray:
    """Equal species split (sizes differ by at most one, larger ones first)."""
    base, rem = divmod(n, n_species)
    sizes = [base + (1 if k < rem else 0) for k in range(n_species)]
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


def frame_from(coords, offsets, box_type, box, r_max, nbins, name="") -> Frame:
    return Frame(np.ascontiguousarray(coords, dtype=np.float32),
                 np.ascontiguousarray(offsets, dtype=np.int64), int(box_type),
                 np.ascontiguousarray(box, dtype=np.float64).reshape(9), float(r_max), int(nbins), name)


def uniform_frame(seed: int, n: int, box_type: int, box: np.ndarray, r_max: float, nbins: int,
                  n_species: int = 1, name: str = "") -> Frame:
    rng = rng_for(seed)
    x = uniform_in_cell(rng, n, box)
    return frame_from(x, even_offsets(n, n_species), box_type, box, r_max, nbins, name)


def config_small_nobox(seed: int = 1, n: int = 2000) -> Frame:
    """Non-periodic, 1 species, N uniform in a cube of side 10, r_max 17.33, 1,000 bins.

    17.33 exceeds the cube diagonal 10*sqrt(3) = 17.3205..., so every pair is in range.
    """
    rng = rng_for(seed)
    x = (rng.random((n, 3)) * 10.0).astype(np.float32)
    return frame_from(x, [0, n], BOX_NONE, np.zeros(9), 17.33, 1000, f"nobox-n{n}")


def config_ortho_two_species(seed: int = 1, n: int = 100_000, side: float = 60.0,
                             r_max: float = 30.0, nbins: int = 10_000) -> Frame:
    """Orthorhombic 60^3 box, N uniform, 2 species of N/2, r_max 30, 10,000 bins."""
    box = ortho_box(side)
    rng = rng_for(seed)
    x = uniform_in_cell(rng, n, box)
    return frame_from(x, even_offsets(n, 2), BOX_ORTHO, box, r_max, nbins, f"ortho2-n{n}")


C3_ANGLES = (70.0, 80.0, 100.0)


def config_triclinic_clusters(seed: int = 1, n: int = 500_000, n_clusters: int = 200,
                              sigma: float = 2.0, background: float = 0.2,
                              r_max: float = 35.0, nbins: int = 20_000,
                              edge: float = 80.0) -> Frame:
    """Triclinic a=b=c=80, alpha=70, beta=80, gamma=100; Gaussian clusters + uniform background.

    A fraction ``background`` of the N particles is uniform in the cell; the rest
    is N(centre, sigma^2 I) around ``n_clusters`` centres uniform in the cell.
    All positions are wrapped into the primary cell, randomly labelled with 3
    species and sorted by label so the species are contiguous.
    """
    box = triclinic_box(edge, edge, edge, *C3_ANGLES)
    rng = rng_for(seed)
    n_bg = int(round(background * n))
    n_cl = n - n_bg
    m = box_matrix(box)
    centres = (m @ rng.random((n_clusters, 3)).T).T
    which = rng.integers(0, n_clusters, size=n_cl)
    pts = centres[which] + rng.normal(0.0, sigma, size=(n_cl, 3))
    bg = (m @ rng.random((n_bg, 3)).T).T
    x = wrap_into_cell(np.concatenate([pts, bg]), box)
    x = x[rng.permutation(n)]
    offsets = even_offsets(n, 3)
    return frame_from(x.astype(np.float32), offsets, BOX_TRICLINIC, box, r_max, nbins,
                      f"tric-clusters-n{n}")


def batch_frames(seed: int = 1, n_frames: int = 256, n_lo: int = 5_000, n_hi: int = 200_000,
                 density: float = 0.1, nbins: int = 4096) -> list[Frame]:
    """Orthorhombic frames with N log-uniform in [n_lo, n_hi], density fixed, species 30/70.

    Box side L = (N/density)^(1/3), r_max = L/2.
    """
    rng = rng_for(seed)
    out = []
    for k in range(n_frames):
        n = int(math.floor(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        side = (n / density) ** (1.0 / 3.0)
        box = ortho_box(side)
        x = uniform_in_cell(rng, n, box)
        na = int(round(0.3 * n))
        out.append(frame_from(x, [0, na, n], BOX_ORTHO, box, side / 2.0, nbins, f"batch{k}-n{n}"))
    return out


def headline_frame(box_type: int, seed: int = 1, n: int = 1_000_000, density: float = 0.1,
                   nbins: int = 10_000) -> Frame:
    """Single-species uniform frame at density 0.1 (N=1M: side 215.44).

    none: cube of the same side, r_max = side*sqrt(3) (every pair in range);
    ortho: cube, r_max = side/2; triclinic: the 70/80/100-degree cell scaled to
    volume N/density, r_max = 0.95 * (smallest plane spacing)/2.
    """
    vol = n / density
    side = vol ** (1.0 / 3.0)
    if box_type == BOX_TRICLINIC:
        box = scale_box(triclinic_box(1.0, 1.0, 1.0, *C3_ANGLES), vol)
        r_max = 0.95 * float(box_heights(box).min()) / 2.0
    else:
        box = ortho_box(side)
        r_max = side / 2.0 if box_type == BOX_ORTHO else side * math.sqrt(3.0)
    rng = rng_for(seed)
    x = uniform_in_cell(rng, n, box)
    f = frame_from(x, [0, n], box_type, box if box_type != BOX_NONE else np.zeros(9), r_max,
                   nbins, f"{BOX_NAMES[box_type]}-n{n}")
    return f


def served_request(rng: np.random.Generator, n_lo: int = 1_000, n_hi: int = 1_000_000,
                   density: float = 0.1) -> Frame:
    """One served request: N log-uniform, box type uniform, 1-3 species, nbins = 2^U{10..14}."""
    n = int(math.floor(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
    box_type = int(rng.integers(0, 3))
    n_species = int(rng.integers(1, 4))
    nbins = 2 ** int(rng.integers(10, 15))
    vol = n / density
    if box_type == BOX_TRICLINIC:
        box = scale_box(triclinic_box(1.0, 1.0, 1.0, *C3_ANGLES), vol)
        r_max = 0.95 * float(box_heights(box).min()) / 2.0
    else:
        side = vol ** (1.0 / 3.0)
        box = ortho_box(side)
        r_max = side / 2.0 if box_type == BOX_ORTHO else side * math.sqrt(3.0)
    x = uniform_in_cell(rng, n, box)
    n_species = min(n_species, n)
    return frame_from(x, even_offsets(n, n_species), box_type,
                      box if box_type != BOX_NONE else np.zeros(9), r_max, nbins,
                      f"req-{BOX_NAMES[box_type]}-n{n}")


def lattice_frame(spacing: float = 0.1, per_side: int = 12, nbins: int = 64,
                  box_type: int = BOX_NONE, jitter_seed: int | None = None) -> Frame:
    """Simple cubic lattice whose spacing equals the bin width (adversarial edge set).

    Many pair distances are then (up to float32 rounding of the positions) exactly
    on bin edges, which exercises the near-edge decision.
    """
    g = np.arange(per_side, dtype=np.float64) * spacing
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    if jitter_seed is not None:
        x = x + rng_for(jitter_seed).normal(0.0, 1e-7, size=x.shape)
    n = x.shape[0]
    side = per_side * spacing
    r_max = nbins * spacing
    box = ortho_box(side) if box_type == BOX_ORTHO else np.zeros(9)
    if box_type == BOX_ORTHO:
        r_max = min(r_max, side / 2.0)
        nbins = int(round(r_max / spacing))
    return frame_from(x.astype(np.float32), [0, n], box_type, box, r_max, nbins,
                      f"lattice-{BOX_NAMES[box_type]}")
