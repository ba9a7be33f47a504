"""The CTA shapes of the sweep variants (csrc/fp_internal.h: sweep_threads, sweep_padded,
sweep_ring, sweep_min_ctas, sweep_has_alt, sweep_batch_shape), evaluated by a small host program
compiled with nvcc, must fit one SM of the GPU for every precision, scheme and switch setting:
the shared memory of the resident CTAs within the SM's 228 KB, the register file (64K) giving
each thread of them at least 64 registers, whole warps, and tiles of 8, 16 and 32 faces that
divide the CTA (the xi pass of an unpadded ring takes 32 faces)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2101_05886_gb300", "csrc")

SM_SHARED = 228 * 1024          # shared memory of one SM (bytes)
CTA_RESERVED = 1024             # reserved per resident CTA
REGISTERS = 65536

PROGRAM = r"""
#include <cstdio>
#include "fp_internal.h"
using namespace fpk;
int main() {
  for (int f32 = 0; f32 < 2; ++f32)
    for (int scheme = 0; scheme < 4; ++scheme)
      for (int fix = 0; fix < 3; ++fix) {
        const int nt = sweep_threads(f32, scheme, fix), ring = sweep_ring(f32, scheme, fix);
        const long long smem = ((long long)(kCellFields + kFaceFields) * ring +
                                (long long)(kNextFields + kEpiFields) * nt) * (f32 ? 4 : 8);
        // static shared memory of the sweep: two block descriptors, two work items, dt and the
        // three global speeds in the state's type, in 16-byte units
        const long long stat = (2 * (long long)sizeof(BlockDev) + 2 * 8 + 4 * (f32 ? 4 : 8) + 15) / 16 * 16;
        std::printf("%d %d %d %d %d %d %d %lld %d %d %lld\n", f32, scheme, fix, nt, (int)sweep_padded(f32, scheme, fix),
                    ring, sweep_min_ctas(f32, scheme, fix), smem, (int)sweep_has_alt(f32, scheme, fix),
                    sweep_batch_shape(f32, scheme, fix), stat);
      }
  return 0;
}
"""


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    return None


@pytest.fixture(scope="module")
def table(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("shapes")
    src, exe = d / "shapes.cu", d / "shapes"
    src.write_text(PROGRAM)
    subprocess.run([nvcc, "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    rows = []
    for line in out.split("\n"):
        if line.strip():
            f32, scheme, fix, nt, pad, ring, minc, smem, alt, bshape, stat = map(int, line.split())
            rows.append(dict(f32=f32, scheme=scheme, fix=fix, nt=nt, pad=pad, ring=ring, minc=minc, smem=smem,
                             alt=alt, bshape=bshape, stat=stat))
    assert len(rows) == 24
    return rows


def test_every_cta_shape_fits_an_sm(table):
    for r in table:
        assert r["nt"] % 32 == 0 and r["nt"] >= 64, r
        assert r["ring"] == (3 if r["pad"] else 2) * r["nt"], r
        assert r["minc"] * (r["smem"] + r["stat"] + CTA_RESERVED) <= SM_SHARED, r
        assert REGISTERS // (r["minc"] * r["nt"]) >= 64, r
        for faces in (8, 16, 32):                        # every tile shape divides the CTA
            assert r["nt"] % faces == 0, r


def test_alternative_shapes_and_batch_choice(table):
    by = {(r["f32"], r["scheme"], r["fix"]): r for r in table}
    for (f32, scheme, fix), r in by.items():
        # an alternative exists only for the folded FP32 sweeps, and it is a different shape
        assert r["alt"] == (f32 == 1 and fix != 0 and scheme <= 2), r
        if r["alt"] and fix == 1:
            assert by[(f32, scheme, 2)]["nt"] != r["nt"], r
        assert r["bshape"] in ((0, 1) if r["alt"] else (0,)), r
    # the measured choices: WENO5 64-thread unpadded CTAs; linear upwind 128 in single blocks,
    # its 64-thread alternative in batches
    assert (by[(1, 0, 1)]["nt"], by[(1, 0, 1)]["pad"], by[(1, 0, 1)]["bshape"]) == (64, 0, 0)
    assert (by[(1, 1, 1)]["nt"], by[(1, 1, 2)]["nt"], by[(1, 1, 1)]["bshape"]) == (128, 64, 1)
