"""Python binding of libdh, the GB300 particle-pair distance histogram library.

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``libdh.so`` (see ``include/dh.h``).  The functions keep the C names
(``dh_create``, ``dh_histogram``, ...); :class:`Context` wraps them for numpy
arrays (host pointers) and torch CUDA tensors (device pointers).  There is no
CPU fallback: if the library has not been built, loading it raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# DH_LIB_PATH selects another build of the same library (for example a debug build)
LIB_PATH = os.environ.get("DH_LIB_PATH") or os.path.join(_HERE, "_lib", "libdh.so")

DH_OK = 0
DH_PENDING = 1
DH_ERR_INVALID = -1
DH_ERR_NOMEM = -2
DH_ERR_CUDA = -3
DH_ERR_TIMEOUT = -4
DH_ERR_CANCELLED = -5
DH_ERR_NOTFOUND = -6

DH_BOX_NONE = 0
DH_BOX_ORTHO = 1
DH_BOX_TRICLINIC = 2

DH_DEVICE_PTRS = 0x1
DH_ACCUMULATE = 0x2
DH_COORDS_F4 = 0x4
DH_COORDS_F64 = 0x8
DH_CFG_NO_GRAPH = 0x1
DH_CFG_TIMING = 0x2
DH_CFG_AUTOTUNE = 0x4
DH_MAX_BINS = 4194240

STATUS_NAMES = {0: "DH_OK", 1: "DH_PENDING", -1: "DH_ERR_INVALID", -2: "DH_ERR_NOMEM",
                -3: "DH_ERR_CUDA", -4: "DH_ERR_TIMEOUT", -5: "DH_ERR_CANCELLED",
                -6: "DH_ERR_NOTFOUND"}


class dh_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("pool_bytes", ctypes.c_uint64),
                ("max_inflight", ctypes.c_int32), ("timeout_ns", ctypes.c_uint64),
                ("tune_cache", ctypes.c_char_p), ("flags", ctypes.c_uint32), ("wave_us", ctypes.c_uint32)]


class dh_frame(ctypes.Structure):
    _fields_ = [("coords", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("species_offsets", ctypes.c_void_p), ("n_species", ctypes.c_int32),
                ("box_type", ctypes.c_int32), ("box", ctypes.c_double * 9),
                ("r_max", ctypes.c_double), ("nbins", ctypes.c_int32),
                ("out", ctypes.c_void_p), ("flags", ctypes.c_uint32)]


class dh_stats(ctypes.Structure):
    _fields_ = [("pairs", ctypes.c_uint64), ("deferred", ctypes.c_uint64),
                ("exact_fallback", ctypes.c_uint64), ("sweeps", ctypes.c_int32),
                ("blocks", ctypes.c_int32), ("items", ctypes.c_int32),
                ("kernel_launches", ctypes.c_int32), ("graph_replays", ctypes.c_int32),
                ("tune_runs", ctypes.c_int32), ("pair_kernel_ms", ctypes.c_double),
                ("tile_j", ctypes.c_int32), ("hist_depth", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("block_threads", ctypes.c_int32),
                ("uniform_pairs", ctypes.c_uint64), ("axis_pairs", ctypes.c_uint64),
                ("warp_agg", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("culled_pairs", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class DHError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None
_lock = threading.Lock()

_SIGNATURES = {
    "dh_create": ([ctypes.POINTER(dh_config), ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "dh_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "dh_set_stream": ([ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "dh_histogram": ([ctypes.c_void_p, ctypes.POINTER(dh_frame)], ctypes.c_int),
    "dh_histogram_async": ([ctypes.c_void_p, ctypes.POINTER(dh_frame)], ctypes.c_int),
    "dh_sync": ([ctypes.c_void_p], ctypes.c_int),
    "dh_histogram_batch": ([ctypes.c_void_p, ctypes.POINTER(dh_frame), ctypes.c_int32], ctypes.c_int),
    "dh_submit": ([ctypes.c_void_p, ctypes.POINTER(dh_frame), ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "dh_poll": ([ctypes.c_void_p, ctypes.c_uint64], ctypes.c_int),
    "dh_wait": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64], ctypes.c_int),
    "dh_cancel": ([ctypes.c_void_p, ctypes.c_uint64], ctypes.c_int),
    "dh_get_stats": ([ctypes.c_void_p, ctypes.POINTER(dh_stats)], ctypes.c_int),
    "dh_last_error": ([ctypes.c_void_p], ctypes.c_char_p),
    "dh_bin_thresholds": ([ctypes.c_double, ctypes.c_int32, ctypes.c_void_p], ctypes.c_int),
    "dh_version": ([], ctypes.c_char_p),
    "dh_selfcheck": ([ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                      ctypes.c_void_p], ctypes.c_int),
    "dh_histogram_noalloc": ([ctypes.POINTER(dh_frame), ctypes.c_void_p], ctypes.c_int),
    "dh_rdf": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p,
                ctypes.c_uint64, ctypes.c_void_p], ctypes.c_int),
    "dh_tune_cache_count": ([ctypes.c_char_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "dh_pipe_rate": ([ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p], ctypes.c_int),
}

DH_NOALLOC_MAX_N = 131072
DH_NOALLOC_MAX_BINS = 65536

PIPES = {"ffma2": 0, "fadd2": 1, "fmul2": 2, "ffma": 3, "sqrt": 4, "frnd": 5, "f2i": 6, "lop3": 7,
         "iadd": 8, "imad": 9, "dfma": 10, "match": 11, "smem_atomic_random": 12,
         "smem_atomic_clustered": 13, "smem_atomic_same": 14, "smem_atomic_sequential": 15,
         "global_atomic64": 16, "dsmem_atomic_c2": 17, "dsmem_atomic_c4": 18, "dsmem_atomic_c8": 19}

DH_CHECK_SQRT = 0
DH_CHECK_WINDOW = 1
DH_CHECK_TILES = 2


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Load libdh.so (raises if it has not been built: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libdh.so not found at {p}: build it with "
                               "`python -m paper_1808_01478_gb300.build`")
        lib = ctypes.CDLL(p)
        for name, (args, res) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        if path is None:
            _lib = lib
        return lib


def exported_symbols() -> list[str]:
    return list(_SIGNATURES)


def _check(status: int, ctx=None) -> int:
    if status < 0:
        msg = load_library().dh_last_error(ctx).decode(errors="replace")
        raise DHError(status, msg)
    return status


# ---------------------------------------------------------------- C-named functions


def dh_version() -> str:
    return load_library().dh_version().decode()


def dh_bin_thresholds(r_max: float, nbins: int) -> np.ndarray:
    out = np.empty(int(nbins) + 1, dtype=np.float64)
    _check(load_library().dh_bin_thresholds(float(r_max), int(nbins), out.ctypes.data_as(ctypes.c_void_p)))
    return out


def dh_tune_cache_count(path: str, sm_count: int) -> int:
    n = ctypes.c_int32(0)
    _check(load_library().dh_tune_cache_count(os.fsencode(path), int(sm_count), ctypes.byref(n)))
    return n.value


def dh_create(device: int = 0, pool_bytes: int = 0, max_inflight: int = 0, timeout_ns: int = 0,
              flags: int = 0, wave_us: int = 0, tune_cache: str | None = None) -> ctypes.c_void_p:
    cfg = dh_config(device, pool_bytes, max_inflight, timeout_ns,
                    None if tune_cache is None else os.fsencode(tune_cache), flags, wave_us)
    h = ctypes.c_void_p()
    _check(load_library().dh_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def dh_destroy(ctx) -> None:
    _check(load_library().dh_destroy(ctx))


def dh_set_stream(ctx, stream_ptr: int | None) -> None:
    _check(load_library().dh_set_stream(ctx, ctypes.c_void_p(stream_ptr or 0)), ctx)


def dh_histogram(ctx, frame: dh_frame) -> None:
    _check(load_library().dh_histogram(ctx, ctypes.byref(frame)), ctx)


def dh_histogram_async(ctx, frame: dh_frame) -> None:
    _check(load_library().dh_histogram_async(ctx, ctypes.byref(frame)), ctx)


def dh_sync(ctx) -> None:
    _check(load_library().dh_sync(ctx), ctx)


def dh_histogram_batch(ctx, frames) -> None:
    arr = (dh_frame * len(frames))(*frames)
    _check(load_library().dh_histogram_batch(ctx, arr, len(frames)), ctx)


def dh_submit(ctx, frame: dh_frame) -> int:
    t = ctypes.c_uint64()
    _check(load_library().dh_submit(ctx, ctypes.byref(frame), ctypes.byref(t)), ctx)
    return int(t.value)


def dh_poll(ctx, ticket: int) -> int:
    return load_library().dh_poll(ctx, ticket)


def dh_wait(ctx, ticket: int, timeout_ns: int) -> int:
    return load_library().dh_wait(ctx, ticket, timeout_ns)


def dh_cancel(ctx, ticket: int) -> int:
    return load_library().dh_cancel(ctx, ticket)


def dh_selfcheck(ctx, what: int, frame: dh_frame | None = None, n_samples: int = 0, seed: int = 0) -> np.ndarray:
    out = np.zeros(4, dtype=np.float64)
    fp = ctypes.byref(frame) if frame is not None else None
    _check(load_library().dh_selfcheck(ctx, int(what), fp, int(n_samples), int(seed),
                                       out.ctypes.data_as(ctypes.c_void_p)), ctx)
    return out


def dh_histogram_noalloc(frame: dh_frame, stream_ptr: int | None = None) -> None:
    """Allocation-free histogram of one frame with device pointers (no context needed)."""
    _check(load_library().dh_histogram_noalloc(ctypes.byref(frame), ctypes.c_void_p(stream_ptr or 0)))


def dh_pipe_rate(device: int, pipe, width: int = 0) -> dict:
    """Measured throughput of one pipe (see dh.h): ops per clock per SM, ops/s, MHz, ms."""
    lib = load_library()
    code = PIPES[pipe] if isinstance(pipe, str) else int(pipe)
    out = (ctypes.c_double * 4)()
    _check(lib.dh_pipe_rate(int(device), code, int(width), out))
    return {"per_clk_sm": out[0], "per_s": out[1], "sm_mhz": out[2], "ms": out[3]}


def dh_rdf(ctx, counts_ptr: int, n_hist: int, nbins: int, r_max: float, pair_density, n_frames: int,
           g_ptr: int) -> None:
    """g(r) of Eq. 1 on the device: counts_ptr (uint64) and g_ptr (double) are device pointers."""
    dens = np.ascontiguousarray(pair_density, dtype=np.float64).reshape(-1)
    if dens.shape[0] != int(n_hist):
        raise ValueError("one pair density per histogram")
    _check(load_library().dh_rdf(ctx, ctypes.c_void_p(counts_ptr), int(n_hist), int(nbins), float(r_max),
                                 dens.ctypes.data_as(ctypes.c_void_p), int(n_frames), ctypes.c_void_p(g_ptr)), ctx)


def dh_get_stats(ctx) -> dict:
    s = dh_stats()
    _check(load_library().dh_get_stats(ctx, ctypes.byref(s)), ctx)
    return s.as_dict()


# ---------------------------------------------------------------- convenience wrapper


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def n_hist(n_species: int) -> int:
    return n_species * (n_species + 1) // 2


class FrameArgs:
    """Keeps the buffers referenced by one dh_frame alive.  float64 coordinates
    (numpy or torch) are passed as binary64 (DH_COORDS_F64), anything else as float32."""

    def __init__(self, coords, offsets, box_type, box, r_max, nbins, out=None, accumulate=False):
        offs = np.ascontiguousarray(offsets, dtype=np.int64)
        s = offs.shape[0] - 1
        self.offsets = offs
        self.keep = [offs]
        flags = 0
        if _is_torch(coords) and coords.is_cuda:
            import torch
            assert coords.dtype in (torch.float32, torch.float64) and coords.is_contiguous()
            if coords.dtype == torch.float64:
                flags |= DH_COORDS_F64
            if coords.dim() == 2 and coords.shape[1] == 4:
                flags |= DH_COORDS_F4
            n = coords.shape[0]
            if out is None:
                out = torch.zeros((n_hist(s), int(nbins)), dtype=torch.int64, device=coords.device)
            assert out.is_cuda and out.is_contiguous() and out.element_size() == 8
            flags |= DH_DEVICE_PTRS
            cptr, optr = coords.data_ptr(), out.data_ptr()
            self.keep += [coords, out]  # the library reads these buffers until the call (or request) ends
        else:
            f64 = np.asarray(coords).dtype == np.float64
            c = np.ascontiguousarray(coords, dtype=np.float64 if f64 else np.float32)
            if f64:
                flags |= DH_COORDS_F64
            if c.ndim == 2 and c.shape[1] == 4:
                flags |= DH_COORDS_F4
            n = c.shape[0]
            if out is None:
                out = np.zeros((n_hist(s), int(nbins)), dtype=np.uint64)
            assert out.flags.c_contiguous and out.dtype.itemsize == 8
            self.keep.append(c)
            cptr = c.ctypes.data if n else 0
            optr = out.ctypes.data if _is_torch(out) is False else out.data_ptr()
        self.coords = coords
        if accumulate:
            flags |= DH_ACCUMULATE
        bx = np.zeros(9) if box is None else np.asarray(box, dtype=np.float64).reshape(9)
        self.out = out
        self.frame = dh_frame(cptr, int(n), offs.ctypes.data, s, int(box_type),
                              (ctypes.c_double * 9)(*bx.tolist()), float(r_max), int(nbins), optr, flags)


class Context:
    """One libdh context (device workspace, stream, threshold cache)."""

    def __init__(self, device: int = 0, **cfg):
        self._inflight = {}
        self.handle = dh_create(device, **cfg)
        self.device = device

    def close(self):
        if self.handle:
            dh_destroy(self.handle)  # cancels and waits for every request still running
            self.handle = None
            self._inflight.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream) -> None:
        ptr = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        dh_set_stream(self.handle, ptr)

    def histogram(self, coords, offsets, box_type, box, r_max, nbins, out=None, accumulate=False):
        fa = FrameArgs(coords, offsets, box_type, box, r_max, nbins, out, accumulate)
        dh_histogram(self.handle, fa.frame)
        return fa.out

    def histogram_frame(self, frame, out=None, device_tensors=None):
        """Histogram of a workloads.Frame (host arrays unless device_tensors=(coords, out))."""
        if device_tensors is not None:
            coords, out = device_tensors
            return self.histogram(coords, frame.offsets, frame.box_type, frame.box, frame.r_max,
                                  frame.nbins, out)
        return self.histogram(frame.coords, frame.offsets, frame.box_type, frame.box, frame.r_max,
                              frame.nbins, out)

    def histogram_async(self, coords, offsets, box_type, box, r_max, nbins, out):
        fa = FrameArgs(coords, offsets, box_type, box, r_max, nbins, out)
        dh_histogram_async(self.handle, fa.frame)
        return fa

    def sync(self):
        dh_sync(self.handle)

    def histogram_batch(self, frame_args: list[FrameArgs]) -> None:
        dh_histogram_batch(self.handle, [fa.frame for fa in frame_args])

    def stats(self) -> dict:
        return dh_get_stats(self.handle)

    def rdf(self, counts, r_max: float, pair_density, n_frames: int):
        """g(r) (torch float64, same shape) from device histograms `counts` (torch
        int64/uint64 viewed as counts, shape (n_hist, nbins) or (nbins,)) summed
        over n_frames frames; pair_density: N_pairs / V per histogram."""
        import torch

        if not (_is_torch(counts) and counts.is_cuda and counts.is_contiguous()):
            raise TypeError("counts must be a contiguous CUDA tensor")
        if counts.dtype not in (torch.int64, torch.uint64):
            raise TypeError("counts must be 64-bit integers")
        c2 = counts.reshape(-1, counts.shape[-1])
        g = torch.empty(counts.shape, dtype=torch.float64, device=counts.device)
        dh_rdf(self.handle, c2.data_ptr(), c2.shape[0], c2.shape[1], r_max, pair_density, n_frames, g.data_ptr())
        return g

    def check_sqrt(self) -> float:
        return float(dh_selfcheck(self.handle, DH_CHECK_SQRT)[0])

    def check_window(self, coords, offsets, box_type, box, r_max, nbins, n_samples=1 << 22, seed=1) -> dict:
        fa = FrameArgs(coords, offsets, box_type, box, r_max, nbins)
        out = dh_selfcheck(self.handle, DH_CHECK_WINDOW, fa.frame, n_samples, seed)
        return {"max_ratio": float(out[0]), "violations": int(out[1]), "checked": int(out[2]),
                "delta": float(out[3])}

    def check_tiles(self, coords, offsets, box_type, box, r_max, nbins, n_tiles=4096, seed=1) -> dict:
        fa = FrameArgs(coords, offsets, box_type, box, r_max, nbins)
        out = dh_selfcheck(self.handle, DH_CHECK_TILES, fa.frame, n_tiles, seed)
        return {"max_ratio": float(out[0]), "violations": int(out[1]), "checked": int(out[2]),
                "shifted_tiles": int(out[3])}

    # served path: the buffers of a submitted request are held here until its
    # final status has been reported (the library reads and writes them until then)
    def submit(self, fa: FrameArgs) -> int:
        t = dh_submit(self.handle, fa.frame)
        self._inflight[t] = fa
        return t

    def _final(self, ticket: int, status: int) -> int:
        if status != DH_PENDING and not (status == DH_ERR_TIMEOUT):
            self._inflight.pop(ticket, None)
        return status

    def poll(self, ticket: int) -> int:
        return self._final(ticket, dh_poll(self.handle, ticket))

    def wait(self, ticket: int, timeout_ns: int = 60_000_000_000) -> int:
        return self._final(ticket, dh_wait(self.handle, ticket, timeout_ns))

    def cancel(self, ticket: int) -> int:
        return dh_cancel(self.handle, ticket)
