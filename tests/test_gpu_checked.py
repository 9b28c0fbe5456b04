"""The bounds-checked build (libgrlb_checked.so, GRLB_CHECKED): every load and store of every
kernel tested against the registry of live device regions.  A battery of small runs through
every kernel family (tests/checked_battery.py: sweeps of every storage x collision on tiled and
linear launches, one-buffer streaming with outflow, Dirichlet tubes with floors, the
Chapman-Enskog start, sources, staging and checkpoints, device-side initialisation, the three
batch schedules and tile shapes, the server, z-slabs, the finiteness scan, the allocation-free
sweep, spectral post-processing, the FFMA probe) runs once on the checked library and once on the
plain one, each in a child process.  Checked: no access outside a live region, every region
released once everything is closed (nothing leaked or released twice), and the checker itself
counts exactly the probe ranges that lie outside.  Both: the same results, bit for bit (the
sweep, initialisation and probe kernels are compiled without multiply-add contraction, every
fused multiply-add being written out, so the checked build's range tests cannot change how an
operation rounds; the spectral kernels keep the compiler's contraction and agree all the same)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2609_16361_b300 import build

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
BATTERY = os.path.join(HERE, "checked_battery.py")


def run_battery(lib, path):
    env = dict(os.environ)
    env.pop("GRLB_LIB", None)
    if lib:
        env["GRLB_LIB"] = lib
    subprocess.run([sys.executable, BATTERY, str(path)], env=env, check=True, timeout=1200)
    with open(path) as f:
        res = json.load(f)
    res["arrays"] = dict(np.load(os.path.splitext(str(path))[0] + ".npz"))
    return res


@pytest.fixture(scope="module")
def runs(tmp_path_factory):
    build.build(checked=True)
    build.build()
    d = tmp_path_factory.mktemp("checked")
    return run_battery(build.LIB_CHECKED, d / "checked.json"), run_battery(None, d / "plain.json")


def test_the_checker_counts_exactly_the_ranges_outside(runs):
    chk, plain = runs
    assert chk["checked"] and not plain["checked"]
    assert len(chk["probe"]) == 7
    for p in chk["probe"]:
        assert p["counted"] == p["expected"], p


def test_every_kernel_access_stays_inside_a_live_region(runs):
    chk, _ = runs
    bad = {k: (v["violations"], hex(v["first"])) for k, v in chk["scenarios"].items() if v["violations"]}
    assert not bad, bad
    assert chk["final"]["violations"] == 0


def test_every_region_is_released_once(runs):
    final = runs[0]["final"]
    assert final["live_regions"] == 0, final
    assert final["unmatched"] == 0 and final["overflow"] == 0, final


def test_checked_results_equal_the_plain_library(runs):
    """Bit for bit, every part of every scenario.  A part that differs is reported with the
    largest difference of each of its arrays relative to the array's magnitude (the size of the
    difference tells a rounding change, ~1e-7, from a wrong access)."""
    chk, plain = runs
    assert set(chk["scenarios"]) == set(plain["scenarios"])
    differ, total = {}, 0
    for name, sc in chk["scenarios"].items():
        pp = plain["scenarios"][name]["parts"]
        assert set(sc["parts"]) == set(pp), name
        for label, v in sc["parts"].items():
            total += 1
            if v["digest"] == pp[label]["digest"]:
                continue
            assert v["narrays"] == pp[label]["narrays"] > 0, (name, label)
            for i in range(v["narrays"]):
                key = f"{name}|{label}|{i}"
                a, b = chk["arrays"][key], plain["arrays"][key]
                differ[key] = float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
    print(f"checked vs plain: {total - len({k.rsplit('|', 1)[0] for k in differ})} of {total} parts bitwise equal")
    assert not differ, "\n".join(f"{k}: {e:.3e}" for k, e in differ.items())
