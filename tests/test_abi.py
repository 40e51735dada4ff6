"""CPU checks of the C ABI: the library loads, exports every declared entry point,
and its host-only logic (the binary64 bin thresholds) agrees with the oracle."""
import os
import re

import numpy as np
import pytest

import paper_1808_01478_gb300 as dh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1808_01478_gb300 import build

    build.build()
    return dh.load_library()


def declared_entry_points():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            text = open(os.path.join(inc, fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(dh_\w+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for required in ("dh_create", "dh_destroy", "dh_histogram", "dh_histogram_batch", "dh_submit",
                     "dh_poll", "dh_wait", "dh_cancel", "dh_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_entry_points():
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    assert dh.dh_version().startswith("dh ")


def test_binding_covers_every_declared_symbol():
    assert set(declared_entry_points()) <= set(dh.exported_symbols())


@pytest.mark.parametrize("r_max,nbins", [(17.33, 1000), (30.0, 10000), (35.0, 20000), (0.1, 1),
                                         (1e-3, 7), (123.456, 4096), (2.0, 3)])
def test_thresholds_agree_with_oracle_bin(lib, oracle_mod, r_max, nbins):
    T = dh.dh_bin_thresholds(r_max, nbins)
    assert T[0] == 0.0
    assert np.all(np.diff(T) > 0)
    ks = range(1, nbins + 1) if nbins <= 1000 else \
        sorted(set(np.random.default_rng(0).integers(1, nbins + 1, 600).tolist()) | {1, nbins})
    for k in ks:
        # T[k] is in bin >= k and the next smaller double is in bin < k
        assert oracle_mod.bin_of(T[k], r_max, nbins) >= k
        assert oracle_mod.bin_of(np.nextafter(T[k], 0.0), r_max, nbins) < k
        # and the threshold is where the edge is expected
        assert abs(np.sqrt(T[k]) - k * r_max / nbins) <= 1e-12 * r_max


def test_thresholds_reject_bad_arguments(lib):
    with pytest.raises(dh.DHError):
        dh.dh_bin_thresholds(0.0, 10)
    with pytest.raises(dh.DHError):
        dh.dh_bin_thresholds(1.0, 0)
    with pytest.raises(dh.DHError):
        dh.dh_bin_thresholds(float("nan"), 10)


def test_tune_cache_file_parsing(lib, tmp_path):
    """The autotuner's cache format: comments, keys for other GPUs and malformed
    lines are skipped, a later line of the same key replaces an earlier one."""
    p = tmp_path / "tune.txt"
    p.write_text("\n".join([
        "# comment line",
        "152 1 14 17 0 1024 256 1 3 1282.4",   # ortho, 10k bins, N ~ 2^17, one frame
        "152 1 14 17 0 512 512 2 2 1290.0",    # same key again: replaces the line above
        "152 0 12 13 3 256 256 4 1 900.5",     # none, 4096 bins, many frames
        "148 2 15 19 0 1024 256 1 3 1000.0",   # another SM count
        "152 2 15 19 0 1000 256 1 3 1000.0",   # tile_j not a power-of-two tile
        "152 2 15 19 0 1024 256 3 3 1000.0",   # depth 3 not offered
        "152 2 15 19 0 1024 256 16 3 1000.0",  # nor depth 16
        "152 2 15 19 0 1024 384 1 3 1000.0",   # block size not offered
        "152 2 15 19 0 1024 2048 1 3 1000.0",  # nor this one
        "152 9 15 19 0 1024 256 1 3 1000.0",   # unknown variant
        "152 2 15 19 0 1024 256 1 3 -1",       # non-positive throughput
        "152 2 15 19 0 1024 1 3 1000.0",       # a field missing
        "152 3 16 20 1 1024 512 1 2 500.0",
        "152 0 10 11 0 1024 256 1 3 20.0 1",   # warp-aggregated increments
        "152 0 10 12 0 1024 512 1 1 20.0 1",   # aggregation needs 256-thread blocks
        "152 0 10 13 0 1024 256 1 3 20.0 2",   # agg is 0 or 1
    ]) + "\n")
    assert dh.dh_tune_cache_count(str(p), 152) == 4
    assert dh.dh_tune_cache_count(str(p), 148) == 1
    assert dh.dh_tune_cache_count(str(p), 132) == 0
    with pytest.raises(dh.DHError) as e:
        dh.dh_tune_cache_count(str(tmp_path / "missing.txt"), 152)
    assert e.value.status == dh.DH_ERR_NOTFOUND


def test_missing_library_fails_loudly(tmp_path):
    # no CPU fallback: without libdh.so the binding raises on first use
    import subprocess
    import sys

    code = ("import paper_1808_01478_gb300 as dh\n"
            "try:\n    dh.Context(0)\nexcept RuntimeError as e:\n    print('raised', e)\n")
    env = dict(os.environ, DH_LIB_PATH=str(tmp_path / "absent" / "libdh.so"))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True,
                         timeout=120)
    assert out.returncode == 0, out.stderr
    assert out.stdout.startswith("raised") and "libdh.so not found" in out.stdout, out.stdout


def test_no_device_fails_loudly(lib):
    # the library is present but no GPU is usable: creating a context returns
    # DH_ERR_CUDA (raised by the binding) instead of computing on the CPU
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(dh.DHError) as e:
        dh.Context(0)
    assert e.value.status == dh.DH_ERR_CUDA


@pytest.mark.parametrize("cname", ["dh_config", "dh_frame", "dh_stats"])
def test_struct_layouts_match_the_header(tmp_path, cname):
    # the ctypes mirrors of the ABI structs against a C compiler's layout of dh.h
    import ctypes
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    py = getattr(dh, cname)
    fields = [name for name, _ in py._fields_]
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "layout.c"
    body = "".join(f'  printf("%zu\\n", offsetof({cname}, {f}));\n' for f in fields)
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "dh.h"\n'
                   f'int main(void) {{\n  printf("%zu\\n", sizeof({cname}));\n{body}  return 0;\n}}\n')
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(root, "include"), str(src), "-o", str(exe)], check=True)
    out = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert out[0] == ctypes.sizeof(py), (cname, out[0], ctypes.sizeof(py))
    for f, off in zip(fields, out[1:]):
        assert getattr(py, f).offset == off, (cname, f, off, getattr(py, f).offset)
