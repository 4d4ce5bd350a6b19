"""The serving loop's admission policy (csrc/admission.h), compiled with a
small C++ driver and run on the CPU: the head request first, then later
requests of the same kind in queue order up to the first that does not
fit, the batch cap, and the other kind left in place."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1702_00339_gb300", "csrc")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("adm") / "admission_driver")
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, os.path.join(ROOT, "tests", "admission_driver.cpp"),
                    "-o", exe], check=True)
    return exe


def _admit(driver, reqs, free, max_batch):
    """reqs: list of (kind, bytes); returns (batch ids, left ids, bytes taken)."""
    lines = [f"{len(reqs)} {free} {max_batch}"] + [f"{k} {b}" for k, b in reqs]
    out = subprocess.run([driver], input="\n".join(lines) + "\n", capture_output=True, text=True,
                         check=True).stdout.strip()
    b, l, t = out.split("|")
    ids = lambda s: [int(x) for x in s.split()[1:]]
    return ids(b), ids(l), int(t)


def test_head_kind_is_batched_in_queue_order(driver):
    reqs = [(0, 10), (1, 10), (0, 10), (1, 10), (0, 10)]
    assert _admit(driver, reqs, 1000, 8) == ([0, 2, 4], [1, 3], 30)
    assert _admit(driver, reqs[1:], 1000, 8) == ([0, 2], [1, 3], 20)   # structured head


def test_first_misfit_of_the_kind_stops_admission(driver):
    reqs = [(0, 10), (1, 5), (0, 100), (0, 10)]
    assert _admit(driver, reqs, 50, 8) == ([0], [1, 2, 3], 10)
    # a request of the other kind never blocks
    reqs = [(0, 10), (1, 10 ** 9), (0, 10)]
    assert _admit(driver, reqs, 50, 8) == ([0, 2], [1], 20)


def test_head_that_does_not_fit_admits_nothing(driver):
    assert _admit(driver, [(1, 60), (1, 10)], 50, 8) == ([], [0, 1], 0)
    assert _admit(driver, [(0, 50)], 50, 8) == ([0], [], 50)            # exactly fits


def test_batch_cap(driver):
    reqs = [(0, 1)] * 6 + [(1, 1)]
    assert _admit(driver, reqs, 1000, 4) == ([0, 1, 2, 3], [4, 5, 6], 4)
    assert _admit(driver, [], 1000, 4) == ([], [], 0)
