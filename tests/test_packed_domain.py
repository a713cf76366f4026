"""The packed tiles' scoring domain and rebase steps, kernel against model.

The bit-level model (``packed16_model``) carries the exactness argument of
the packed 16-bit tiles: which scorings they hold and how far the frame is
rebased.  The kernel header decides the same two things on the host when it
routes a scoring (packed16_ok, packed32_ok, rebase_step16).  This test
compiles those host-side functions from ``xd_lockstep16.cuh`` with nvcc
(no GPU needed), evaluates them over a grid of scorings that crosses every
limit, and requires them to equal the model's, so that the argument the
model pins is the one the kernel relies on.
"""
import os
import shutil
import subprocess

import pytest

import packed16_model as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MATCH = [1, 2, 3, 7, 64, 126, 127, 128]
GAP = [-1, -2, -3, -64, -125, -127, -128]
MISMATCH = [0, -1, -2, -3, -127, -128, -129]
X = [0, 1, 50, 509, 510, 1020, 1021, 1022, 1023, 1534, 1535, 1536]

PROGRAM = r"""
#include <stdio.h>
#include "xd_lockstep16.cuh"
int main(void)
{
    const int match[] = {%(match)s}, gap[] = {%(gap)s}, mis[] = {%(mis)s}, x[] = {%(x)s};
    for (int a : match) for (int g : gap) for (int b : mis) for (int c : x) {
        const xd::Scoring sc{a, b, g, c};
        printf("%%d %%d %%d %%d %%d %%d %%d %%d\n", a, b, g, c, (int)xd::packed16_ok(sc),
               (int)xd::packed32_ok(sc), xd::rebase_step16<16>(sc), xd::rebase_step16<32>(sc));
    }
    return 0;
}
"""


def test_kernel_domain_and_rebase_steps_equal_the_model(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("no nvcc")
    src = tmp_path / "domain.cu"
    src.write_text(PROGRAM % {"match": ", ".join(map(str, MATCH)), "gap": ", ".join(map(str, GAP)),
                              "mis": ", ".join(map(str, MISMATCH)), "x": ", ".join(map(str, X))})
    exe = tmp_path / "domain"
    csrc = os.path.join(ROOT, "paper_2309_07270_gb300", "csrc")
    subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I", csrc,
                    "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    rows = [list(map(int, ln.split())) for ln in out if ln]
    assert len(rows) == len(MATCH) * len(GAP) * len(MISMATCH) * len(X)
    n16 = n32 = 0
    for m, mis, g, x, ok16, ok32, k16, k32 in rows:
        assert bool(ok16) == P.fits(m, mis, g, x, 16), (m, mis, g, x)
        assert bool(ok32) == P.fits(m, mis, g, x, 32), (m, mis, g, x)
        if ok16:
            n16 += 1
            assert k16 == P.rebase_step(m, g, x, 16), (m, g, x)
        if ok32:
            n32 += 1
            assert k32 == P.rebase_step(m, g, x, 32), (m, g, x)
    # the grid reaches both sides of every limit
    assert 0 < n32 < n16 < len(rows)
