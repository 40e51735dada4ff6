"""FP64 CPU oracle for the particle-pair distance histogram (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never calls it and
shares no code with it.  The arithmetic lives in ``dh_oracle.cpp`` (plain C++,
binary64, no contraction); this module only compiles that file and marshals
numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(_HERE, "dh_oracle.cpp")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libdh_oracle.so")
_lock = threading.Lock()
_default = None

# -O2 without -ffast-math; -ffp-contract=off keeps every binary64 operation as
# written (no implicit fused multiply-add).
CXXFLAGS = ["-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
            "-fopenmp"]


def _compile(src_path: str, out_path: str) -> None:
    os.makedirs(os.path.dirname(out_path), exist_ok=True)
    tmp = out_path + f".tmp{os.getpid()}"
    subprocess.run(["g++", *CXXFLAGS, src_path, "-o", tmp], check=True)
    os.replace(tmp, out_path)


def build(force: bool = False) -> str:
    """Compile the oracle shared library (g++) if missing or stale; return its path."""
    if (force or not os.path.exists(_LIB_PATH)
            or os.path.getmtime(_LIB_PATH) < os.path.getmtime(SRC)):
        _compile(SRC, _LIB_PATH)
    return _LIB_PATH


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _box9(box) -> np.ndarray:
    return np.ascontiguousarray(box if box is not None else np.zeros(9), dtype=np.float64).reshape(9)


class OracleLib:
    """ctypes view of one compiled oracle library."""

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        lib.dh_oracle_histogram.argtypes = [P, ctypes.c_int64, P, ctypes.c_int32, ctypes.c_int32,
                                            P, ctypes.c_double, ctypes.c_int32, P, ctypes.c_int32]
        lib.dh_oracle_histogram.restype = ctypes.c_int
        lib.dh_oracle_histogram_f64.argtypes = lib.dh_oracle_histogram.argtypes
        lib.dh_oracle_histogram_f64.restype = ctypes.c_int
        lib.dh_oracle_pair_r2.argtypes = [P, P, ctypes.c_int32, P]
        lib.dh_oracle_pair_r2.restype = ctypes.c_double
        lib.dh_oracle_bin.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int32]
        lib.dh_oracle_bin.restype = ctypes.c_int64
        lib.dh_oracle_pairs_r2.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_int32, P, P]
        lib.dh_oracle_pairs_r2.restype = None
        lib.dh_oracle_pairs_r2_f64.argtypes = lib.dh_oracle_pairs_r2.argtypes
        lib.dh_oracle_pairs_r2_f64.restype = None
        lib.dh_oracle_rdf.argtypes = [P, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, P, ctypes.c_uint64, P]
        lib.dh_oracle_rdf.restype = None
        lib.dh_oracle_histogram_one.argtypes = [P, ctypes.c_int64, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                 ctypes.c_int32, P, ctypes.c_double, ctypes.c_int32, P,
                                                 ctypes.c_int32]
        lib.dh_oracle_histogram_one.restype = ctypes.c_int
        lib.dh_oracle_max_threads.argtypes = []
        lib.dh_oracle_max_threads.restype = ctypes.c_int
        self.lib = lib
        self.path = path

    def max_threads(self) -> int:
        return int(self.lib.dh_oracle_max_threads())

    def histogram(self, coords, offsets, box_type, box, r_max, nbins,
                  nthreads: int | None = None) -> np.ndarray:
        """All S(S+1)/2 species-pair histograms, shape (S(S+1)/2, nbins), uint64.
        float64 coordinates use the binary64-input definition, anything else float32."""
        f64 = np.asarray(coords).dtype == np.float64
        x = np.ascontiguousarray(coords, dtype=np.float64 if f64 else np.float32).reshape(-1, 3)
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        bx = _box9(box)
        s = off.shape[0] - 1
        out = np.zeros((s * (s + 1) // 2, int(nbins)), dtype=np.uint64)
        nt = self.max_threads() if nthreads is None else int(nthreads)
        fn = self.lib.dh_oracle_histogram_f64 if f64 else self.lib.dh_oracle_histogram
        rc = fn(_ptr(x), x.shape[0], _ptr(off), s, int(box_type), _ptr(bx), float(r_max), int(nbins), _ptr(out), nt)
        if rc != 0:
            raise ValueError(f"oracle rejected the frame (code {rc})")
        return out

    def histogram_one(self, coords, offsets, box_type, box, r_max, nbins, a: int, c: int,
                      nthreads: int | None = None) -> np.ndarray:
        """The histogram of species pair (a, c), a <= c, alone (float32 coordinates), shape (nbins,)."""
        x = np.ascontiguousarray(coords, dtype=np.float32).reshape(-1, 3)
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        bx = _box9(box)
        out = np.zeros(int(nbins), dtype=np.uint64)
        nt = self.max_threads() if nthreads is None else int(nthreads)
        rc = self.lib.dh_oracle_histogram_one(_ptr(x), x.shape[0], _ptr(off), off.shape[0] - 1, int(a), int(c),
                                              int(box_type), _ptr(bx), float(r_max), int(nbins), _ptr(out), nt)
        if rc != 0:
            raise ValueError(f"oracle rejected the frame (code {rc})")
        return out

    def histogram_frame(self, frame, nthreads: int | None = None) -> np.ndarray:
        return self.histogram(frame.coords, frame.offsets, frame.box_type, frame.box, frame.r_max,
                              frame.nbins, nthreads)

    def pair_r2(self, xi, xj, box_type, box) -> float:
        a = np.ascontiguousarray(xi, dtype=np.float32).reshape(3)
        b = np.ascontiguousarray(xj, dtype=np.float32).reshape(3)
        bx = _box9(box)
        return float(self.lib.dh_oracle_pair_r2(_ptr(a), _ptr(b), int(box_type), _ptr(bx)))

    def pairs_r2(self, coords, ii, jj, box_type, box) -> np.ndarray:
        f64 = np.asarray(coords).dtype == np.float64
        x = np.ascontiguousarray(coords, dtype=np.float64 if f64 else np.float32).reshape(-1, 3)
        i = np.ascontiguousarray(ii, dtype=np.int64)
        j = np.ascontiguousarray(jj, dtype=np.int64)
        bx = _box9(box)
        out = np.empty(i.shape[0], dtype=np.float64)
        fn = self.lib.dh_oracle_pairs_r2_f64 if f64 else self.lib.dh_oracle_pairs_r2
        fn(_ptr(x), _ptr(i), _ptr(j), i.shape[0], int(box_type), _ptr(bx), _ptr(out))
        return out

    def bin_of(self, r2: float, r_max: float, nbins: int) -> int:
        return int(self.lib.dh_oracle_bin(float(r2), float(r_max), int(nbins)))

    def rdf(self, counts, r_max: float, pair_density, n_frames: int) -> np.ndarray:
        """g(r) of Eq. 1 per bin from histograms summed over n_frames frames;
        pair_density[h] = N_pairs / V of histogram h."""
        c = np.ascontiguousarray(counts, dtype=np.uint64)
        c2 = c.reshape(-1, c.shape[-1])
        dens = np.ascontiguousarray(pair_density, dtype=np.float64).reshape(-1)
        if dens.shape[0] != c2.shape[0]:
            raise ValueError("one pair density per histogram")
        g = np.empty(c2.shape, dtype=np.float64)
        self.lib.dh_oracle_rdf(_ptr(c2), c2.shape[0], c2.shape[1], float(r_max), _ptr(dens), int(n_frames),
                               _ptr(g))
        return g.reshape(c.shape)


def default() -> OracleLib:
    global _default
    with _lock:
        if _default is None:
            _default = OracleLib(build())
    return _default


def build_variant(source_text: str, tag: str) -> OracleLib:
    """Compile a modified copy of the oracle source (used to plant mistakes in tests)."""
    src = os.path.join(_BUILD_DIR, f"variant_{tag}.cpp")
    os.makedirs(_BUILD_DIR, exist_ok=True)
    with open(src, "w") as fh:
        fh.write(source_text)
    out = os.path.join(_BUILD_DIR, f"libvariant_{tag}.so")
    _compile(src, out)
    return OracleLib(out)


def max_threads() -> int:
    return default().max_threads()


def histogram(coords, offsets, box_type, box, r_max, nbins, nthreads: int | None = None):
    return default().histogram(coords, offsets, box_type, box, r_max, nbins, nthreads)


def histogram_one(coords, offsets, box_type, box, r_max, nbins, a: int, c: int, nthreads: int | None = None):
    return default().histogram_one(coords, offsets, box_type, box, r_max, nbins, a, c, nthreads)


def histogram_frame(frame, nthreads: int | None = None):
    return default().histogram_frame(frame, nthreads)


def pair_r2(xi, xj, box_type, box) -> float:
    return default().pair_r2(xi, xj, box_type, box)


def pairs_r2(coords, ii, jj, box_type, box):
    return default().pairs_r2(coords, ii, jj, box_type, box)


def bin_of(r2: float, r_max: float, nbins: int) -> int:
    return default().bin_of(r2, r_max, nbins)


def rdf(counts, r_max: float, pair_density, n_frames: int):
    return default().rdf(counts, r_max, pair_density, n_frames)
