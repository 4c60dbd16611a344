"""The blocked c2c layout's line mapping (blocked_line in csrc/afft_internal.h), compiled for the
host with nvcc and checked on the CPU: it is a permutation of the lines; a CTA's run of lines
(its count dividing the 32-line block) stays consecutive, so the contiguous stage remaps only its
first line; the N0 stage's [(n1/32) batch][n0][32 n2] view and the N1 stage's 4-D map
[n1/32][batch n0][32][n2] (row r of block k of plane o at line (k batch n0 + o) 32 + r) address
exactly the lines the mapping gives.  Also that stage_order (the alternating tile order of
consecutive stages) visits every tile once, first to last or last to first."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_1506_07933_gb300", "csrc", "afft_internal.h")

PROGRAM = r'''
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "%s"
using namespace afft;
// argv: n0 n1 n2 batch lines; prints "ok" or the first failure
int main(int argc, char **argv)
{
    const long long n0 = atoll(argv[1]), n1 = atoll(argv[2]), n2 = atoll(argv[3]), B = atoll(argv[4]);
    const int lines = atoi(argv[5]), blk = 32;
    StageDesc d{};
    d.blk = blk; d.blk_in = 0; d.blk_out = 1; d.blk_n1 = n1; d.blk_planes = B * n0;
    const long long P0 = B * n0, nl = P0 * n1;
    std::vector<char> hit(nl, 0);
    for (long long q = 0; q < nl; ++q) {
        const long long t = blocked_line(d, q);
        if (t < 0 || t >= nl || hit[t]) { printf("not a permutation at %%lld\n", q); return 1; }
        hit[t] = 1;
    }
    for (long long b0 = 0; b0 < nl; b0 += lines)
        for (long long i = 1; i < lines && b0 + i < nl; ++i)
            if (blocked_line(d, b0 + i) != blocked_line(d, b0) + i) { printf("run broken at %%lld\n", b0); return 1; }
    const long long W0 = blk * n2;
    for (long long pl = 0; pl < P0; ++pl)
        for (long long j = 0; j < n1; ++j) {
            const long long bt = pl / n0, i0 = pl %% n0;
            const long long o = (j / blk) * B + bt;                      // N0 view: outer line o, row i0
            if ((o * n0 + i0) * W0 + (j %% blk) * n2 != blocked_line(d, pl * n1 + j) * n2) {
                printf("N0 view at plane %%lld line %%lld\n", pl, j); return 1;
            }
            const long long z = (j / blk) * P0 + pl;                     // N1 map: block j / 32, plane pl
            if (z * blk + j %% blk != blocked_line(d, pl * n1 + j)) { printf("N1 box at %%lld %%lld\n", pl, j); return 1; }
        }
    // the alternating stage order walks every tile once: first to last, or last to first
    for (long long n = 1; n <= 400; n += 37)
        for (int rev = 0; rev < 2; ++rev) {
            std::vector<char> seen(n, 0);
            for (long long i = 0; i < n; ++i) {
                const long long t = stage_order(i, n, rev);
                if (t < 0 || t >= n || seen[t] || t != (rev ? n - 1 - i : i)) {
                    printf("stage order %%lld of %%lld (rev %%d)\n", i, n, rev); return 1;
                }
                seen[t] = 1;
            }
        }
    printf("ok\n");
    return 0;
}
'''


@pytest.fixture(scope="module")
def layout_prog(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("layout")
    src, exe = str(d / "layout.cu"), str(d / "layout")
    with open(src, "w") as fh:
        fh.write(PROGRAM % HEADER)
    subprocess.check_call([nvcc, "-std=c++17", "-O1", "-o", exe, src])
    return exe


@pytest.mark.parametrize("n0,n1,n2,batch,lines", [(64, 64, 256, 1, 16), (16, 64, 128, 3, 32), (24, 64, 1024, 2, 2),
                                                  (96, 32, 512, 3, 8), (1024, 64, 1024, 1, 4),
                                                  (512, 32, 128, 1, 32), (8, 96, 4096, 2, 1)])
def test_blocked_line_mapping(layout_prog, n0, n1, n2, batch, lines):
    r = subprocess.run([layout_prog, str(n0), str(n1), str(n2), str(batch), str(lines)],
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout
