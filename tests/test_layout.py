"""Host-side invariants of the per-world shared-memory layout (kamino_internal.h), checked by
compiling the header with the host compiler: every phase's scratch fits the region it is given,
the panel stride keeps the tensor-core fragment loads conflict-free and grows with the row count,
offsets are 16-byte aligned, and the biped / heightfield layouts fit the 227 KB a CTA may use."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2603_16536_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "kamino_internal.h"
using namespace kamino;
static size_t field_ok(const Layout &L) {
    const size_t f[] = {L.bq, L.bu, L.bRd, L.bI, L.bIinv, L.bminv, L.bufree, L.jwr, L.cid, L.cslot, L.rbody,
                        L.rJ, L.rvs, L.rreg, L.lgap, L.lJ, L.lrank, L.lcid, L.vfd, L.p, L.x, L.xn, L.y, L.z, L.yh, L.zh, L.b, L.mut, L.mui, L.wv, L.fb,
                        L.bro, L.brow, L.X, L.A, L.red, L.misc};
    for (size_t o : f) if (o % 16) return 0;
    return 1;
}
int main() {
    int bad = 0;
    for (int mp = 16; mp <= kMaxRowsPad; mp += 16) {
        const int ld = panel_ld(mp);
        if (ld < mp || ld % 32 != 8) { printf("panel_ld %d -> %d\n", mp, ld); ++bad; }
        if (mp > 16 && ld < panel_ld(mp - 16)) { printf("panel_ld not monotone at %d\n", mp); ++bad; }
        for (int nbp : {8, 16})
            for (int nb : {1, 3, 13, 31, 64}) {
                const Layout L = make_layout<float>(nb, 36, 32, mp, nbp);
                const size_t xs = (L.A - L.X) / sizeof(float);
                const size_t need_sweep = 2 * (size_t)ld * nbp + (size_t)nbp * nbp;
                const size_t need_rows = 12 * (size_t)mp;
                const size_t need_refine = (size_t)kWarps * mp + 2 * (size_t)mp + 12 * (size_t)nb;
                if (xs < need_sweep || xs < need_rows || xs < need_refine) {
                    printf("X too small: mp %d nb %d nbp %d\n", mp, nb, nbp); ++bad;
                }
                if (L.A + (size_t)mp * (mp + 1) / 2 * sizeof(float) > L.red) { printf("A overlaps\n"); ++bad; }
                if (!field_ok(L)) { printf("misaligned field: mp %d\n", mp); ++bad; }
                const Layout D = make_layout<double>(nb, 36, 32, mp, nbp);
                if (!field_ok(D)) { printf("misaligned field (double): mp %d\n", mp); ++bad; }
            }
    }
    // the benchmark's worlds: biped (31 bodies, 36 joints, 16 candidates, 240 padded rows, panel 16)
    // and the heightfield biped (32 candidates, 288 padded rows, panel 8)
    const size_t biped = make_layout<float>(31, 36, 16, 240, 16).total;
    const size_t hf = make_layout<float>(31, 36, 32, 288, 8).total;
    printf("biped %zu heightfield %zu\n", biped, hf);
    if (biped > 232448 || hf > 232448) ++bad;
    // the sweep in tensor memory stages two 256-row K-major panels and the pivot block in X
    const Layout L = make_layout<float>(31, 36, 16, 240, 16);
    if ((L.A - L.X) < (2 * 256 * 16 + 256) * sizeof(float)) { printf("no room for the TMEM sweep panels\n"); ++bad; }
    return bad;
}
"""


def test_shared_memory_layout_invariants(tmp_path):
    cxx = shutil.which("g++")
    cuda_inc = "/usr/local/cuda/include"
    if cxx is None or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    src = tmp_path / "layout.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "layout"
    subprocess.run([cxx, "-std=c++17", "-O1", f"-I{CSRC}", f"-I{os.path.join(ROOT, 'include')}", f"-I{cuda_inc}",
                    str(src), "-o", str(exe)], check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout
