"""The library's real-coordinate index maps against the oracle's coordinate
order (oracle.hermitian: the diagonal, then Re and Im of the upper-triangle
entries in row-major order).  herm_coord (coordinate -> (k, l, part)) is
computed in closed form from the root of a quadratic, corrected by whole
steps; herm_pair_coord ((k, l) -> coordinate) from the number of pairs
before row k.  Both are host-and-device code of lb_internal.cuh, compiled
here into a host-only program (nvcc, no GPU needed) and checked for every
coordinate at d = 1 .. 12, 27, 64 and 181."""

import os
import shutil
import subprocess
import tempfile

import pytest

from oracle.hermitian import pairs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DS = list(range(1, 13)) + [27, 64, 181]


def _nvcc():
    for c in (os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc"), shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    return None


@pytest.fixture(scope="module")
def maps():
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "herm_coords")
        cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O1",
               "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_2603_18052_gb300", "csrc"),
               os.path.join(ROOT, "tests", "herm_coords_main.cu"), "-o", exe]
        subprocess.run(cmd, check=True, capture_output=True)
        out = subprocess.run([exe] + [str(d) for d in DS], check=True, capture_output=True, text=True).stdout
    res, d = {}, None
    for line in out.splitlines():
        f = line.split()
        if f[0] == "d":
            d = int(f[1])
            res[d] = {"c": {}, "p": {}}
        elif f[0] == "c":
            res[d]["c"][int(f[1])] = (int(f[2]), int(f[3]), int(f[4]))
        else:
            res[d]["p"][(int(f[1]), int(f[2]))] = int(f[3])
    return res


@pytest.mark.parametrize("d", DS)
def test_coordinate_maps_follow_the_oracle_order(maps, d):
    m = maps[d]
    want = {a: (a, a, 0) for a in range(d)}
    for q, (k, l) in enumerate(pairs(d)):
        want[d + 2 * q] = (k, l, 1)
        want[d + 2 * q + 1] = (k, l, 2)
        assert m["p"][(k, l)] == d + 2 * q
    assert m["c"] == want
    assert len(m["p"]) == d * (d - 1) // 2
