"""The oracle against the hand-worked histograms of tests/golden/hand_cases.txt
(each case derived on paper from Alg. 1, Eq. 4 and Eq. 5; see the file)."""
import os

import numpy as np
import pytest

import workloads as w

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "hand_cases.txt")
BOX = {"none": w.BOX_NONE, "ortho": w.BOX_ORTHO, "triclinic": w.BOX_TRICLINIC}


def load_cases(path):
    cases, cur, mode = [], None, None
    for raw in open(path):
        line = raw.strip()
        if not line or line.startswith("#"):
            continue
        key, _, rest = line.partition(" ")
        if key == "case":
            cur = {"name": rest, "box": np.zeros(9), "coords": [], "expect": []}
            mode = None
        elif key in ("coords", "expect"):
            mode = key
        elif key == "end":
            cases.append(cur)
            cur, mode = None, None
        elif mode is not None:
            cur[mode].append([float(v) for v in line.split()])
        elif key == "box_type":
            cur["box_type"] = BOX[rest]
        elif key == "box":
            cur["box"] = np.array([float(v) for v in rest.split()])
        elif key == "r_max":
            cur["r_max"] = float(rest)
        elif key == "nbins":
            cur["nbins"] = int(rest)
        elif key == "offsets":
            cur["offsets"] = [int(v) for v in rest.split()]
        else:
            raise ValueError(f"unknown key {key!r} in {path}")
    return cases


CASES = load_cases(GOLDEN)


def test_fixture_is_well_formed():
    assert len(CASES) >= 7
    for c in CASES:
        s = len(c["offsets"]) - 1
        assert c["offsets"][-1] == len(c["coords"]), c["name"]
        assert len(c["expect"]) == s * (s + 1) // 2, c["name"]
        assert all(len(h) == c["nbins"] for h in c["expect"]), c["name"]


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_oracle_reproduces_hand_worked_histograms(oracle_mod, case):
    x = np.array(case["coords"], dtype=np.float32)
    got = oracle_mod.histogram(x, case["offsets"], case["box_type"], case["box"], case["r_max"], case["nbins"])
    want = np.array(case["expect"], dtype=np.uint64)
    assert np.array_equal(got, want), (case["name"], got.tolist())
