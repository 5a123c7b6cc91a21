"""Shared-memory layouts of the kernels (host arithmetic in csrc/kt_internal.h).

The occupancy the kernels are designed for rests on these byte counts: the lean
FP32-LU lane layout must fit eight warps of 11 unknowns beside the combustion network's
staged tables in one SM's 227 KB, the Jacobian-cache layout four; the warp kernels'
TR-BDF2 layout (Jacobian in the iteration matrix's storage) must fit four warps of the
64-species network beside its 53 KB of staged tables.  Compiled with the host compiler
only; no GPU.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2504_04941_gb300", "csrc")
SMEM_OPTIN = 232448          # 227 KB of dynamic shared memory per block on this GPU

PROBE = r"""
#include <cstdio>
#include "kt_internal.h"
int main(int argc, char **argv)
{
    (void)argc;
    const int blob = std::atoi(argv[1]), blob_warp = std::atoi(argv[2]);
    const kt::LaneLayout lean = kt::lane_layout_lean(11, 60, 1, blob, 0);
    const kt::LaneLayout jc = kt::lane_layout(11, 60, 1, 1, blob, 0, 0);
    const kt::LaneLayout lean3 = kt::lane_layout_lean(3, 3, 0, 2560, 0);
    const kt::WarpLayout w_tr = kt::warp_layout(65, 1000, 1, 1, blob_warp, true);
    const kt::WarpLayout w_be = kt::warp_layout(65, 1000, 1, 1, blob_warp, false);
    std::printf("%d %d %d %d %d %d %d %d %d %d %d %d\n", lean.base, lean.warp_bytes, jc.base, jc.warp_bytes,
                lean3.base, lean3.warp_bytes, w_tr.base, w_tr.warp_bytes, w_be.warp_bytes, w_tr.off_J,
                w_tr.off_M, lean.off_V == lean.off_W);
    return 0;
}
"""


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("layouts")
    src, exe = d / "probe.cpp", d / "probe"
    src.write_text(PROBE)
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, "-include", "cstdlib", str(src), "-o", str(exe)],
                   check=True, capture_output=True)

    def run(blob, blob_warp):
        out = subprocess.run([str(exe), str(blob), str(blob_warp)], check=True, capture_output=True, text=True)
        return [int(x) for x in out.stdout.split()]
    return run


def test_lane_layouts_fit_the_designed_warps(probe):
    # the combustion network's staged tables: ~7.4 KB (rates, indices, FP32 copies, lists, exp table)
    lean_base, lean_w, jc_base, jc_w, l3_base, l3_w, *_ = probe(7392, 53248)
    assert lean_w == 27136                                   # 11 unknowns, lean: 27,136 B per warp
    assert lean_base + 8 * lean_w <= SMEM_OPTIN               # eight warps per block fit
    assert jc_w > 2 * 25000 and jc_base + 4 * jc_w <= SMEM_OPTIN < jc_base + 5 * jc_w
    assert l3_base + 8 * l3_w <= SMEM_OPTIN                   # Robertson, lean


def test_warp_layout_tr_shares_the_jacobian_storage(probe):
    *_, w_base, w_tr, w_be, off_j, off_m, v_over_w = probe(7392, 53248)
    assert off_j == off_m and v_over_w == 1
    nn = 65 * 65 * 4
    assert w_be - w_tr >= nn - 16                             # one 65 x 65 FP32 matrix less
    assert w_base + 4 * w_tr <= SMEM_OPTIN < w_base + 4 * w_be
