"""Host check of the rasterizer's per-scanline arithmetic with Sec. 4.1.1's
merge (paper_2602_07782_gb300/csrc/raster_math.cuh compiled with g++): the
constants of a chart at a scale -- its slices along the axis (pieces), the
slices of the other axis (cross pieces) and the OBB lines and corners, the
corners taken at any scale by one division as the prefix-sum tail does --
give, scanline by scanline, the oracle's unpadded TopEdge/BottomEdge and
left/right extents.  The chart records come from the CPU oracle (ten slots
per axis, slot t holding slice floor(t K / 10)); the GPU parity tests check
the rasterizer itself."""
from __future__ import annotations

import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <cstdio>
#include <cstdint>
#include <cmath>
#include "raster_math.cuh"
using namespace tabi::rmath;

// one chart per input line: Wq Hq m u0 u1 v0 v1 K use_l use_o k, then the
// ten slots of ylo, yhi, xlo, xhi; prints the raw column bounds, then the
// raw row bounds
int main() {
  long long Wq, Hq, m, u0, u1, v0, v1, K, ul, uo, k;
  while (std::scanf("%lld %lld %lld %lld %lld %lld %lld %lld %lld %lld %lld", &Wq, &Hq, &m, &u0, &u1, &v0, &v1, &K,
                    &ul, &uo, &k) == 11) {
    long long sl[4][10];
    for (int a = 0; a < 4; ++a)
      for (int i = 0; i < 10; ++i) std::scanf("%lld", &sl[a][i]);
    const int64_t C = llround(16384.0 * cos(m * 3.14159265358979323846 / 16.0));
    const int64_t S = llround(16384.0 * sin(m * 3.14159265358979323846 / 16.0));
    AxisK ax[2];
    for (int a = 0; a < 2; ++a) {
      const uint32_t ext = (uint32_t)(a ? Hq : Wq), oth = (uint32_t)(a ? Wq : Hq);
      for (int i = 0; i < 10; ++i) {
        const int s = i * (int)K / 10;
        setup_piece(ax[a], i, i * ext / 10, (i + 1) * ext / 10, (uint32_t)k, (uint32_t)(a ? sl[2][i] : sl[0][i]),
                    (uint32_t)(a ? sl[3][i] : sl[1][i]));
        setup_cross(ax[a], i, (uint32_t)(a ? sl[0][i] : sl[2][i]), (uint32_t)(a ? sl[1][i] : sl[3][i]), ext,
                    (uint32_t)k, (uint32_t)(s * 10 / K) * oth / 10, (uint32_t)((s + 1) * 10 / K) * oth / 10);
      }
      const Magic qC = magic_div((uint32_t)C), qS = magic_div(S > 1 ? (uint32_t)S : 2u);
      setup_obb_fixed(ax[a], a, (int)m, C, S, qC, qS, ul != 0, uo != 0);
      setup_obb_k(ax[a], a, Wq, Hq, k, C, S, u0, u1, v0, v1);
      if (ax[a].use_o)
        for (int it = 0; it < 4; ++it) {
          CornerQ cq;
          corner_at(cq, a * 4 + it, k, C, S, u0, u1, v0, v1);
          corner_store(cq, a * 4 + it, ax[a], (a ? Hq : Wq) * k);
        }
    }
    for (int a = 0; a < 2; ++a) {
      for (int c = 0; c < ax[a].len; ++c) {
        int32_t lo, hi;
        scanline(ax[a], c, lo, hi);
        std::printf("%d %d ", lo, hi);
      }
      std::printf("\n");
    }
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def exe():
    with tempfile.TemporaryDirectory() as td:
        src = os.path.join(td, "t.cpp")
        out = os.path.join(td, "t")
        with open(src, "w") as f:
            f.write(PROGRAM)
        inc = os.path.join(ROOT, "paper_2602_07782_gb300", "csrc")
        r = subprocess.run(["g++", "-O2", "-std=c++17", "-I", inc, src, "-o", out], capture_output=True, text=True)
        if r.returncode != 0:
            pytest.fail(r.stderr[-3000:])
        yield out


@pytest.mark.parametrize("kk", [10, 5, 2])
@pytest.mark.parametrize("flags", [oracle.F_ALL, oracle.F_ALL & ~oracle.F_OBB, oracle.F_ALL & ~oracle.F_LAABB])
def test_scanlines_match_the_oracle(exe, kk, flags):
    R = oracle.R
    cs = synth.knees(3, 60, 512)
    T = 256
    stair = [(0, 0), (6 * T, 0), (6 * T, 10 * T), (8 * T, 10 * T), (8 * T, 16 * T), (0, 16 * T)]
    cs2 = synth.from_polygons([stair], 64, 64)
    params = oracle.default_params(laabb_k=kk, flags=flags)
    lines, want = [], []
    rng = np.random.default_rng(kk * 100 + flags)
    for c_set in (cs, cs2):
        rec = oracle.prep(c_set, params)
        for r in rec:
            for k in [int(v) for v in rng.integers(1, 1025, 3)] + [1024, 512]:
                slots = [[int(r[R[f] + t * kk // 10]) for t in range(10)] for f in ("YLO", "YHI", "XLO", "XHI")]
                head = [int(r[R[f]]) for f in ("WQ", "HQ", "OBBM", "U0", "U1", "V0", "V1")]
                lines.append(" ".join(str(v) for v in head + [kk, int((flags & oracle.F_LAABB) != 0),
                                                                int((flags & oracle.F_OBB) != 0), k] +
                                      sum(slots, [])))
                e = oracle.envelope(r, k, params)
                want.append((np.stack([e.top, e.bot], 1).ravel(), np.stack([e.left, e.right], 1).ravel()))
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, timeout=300)
    assert out.returncode == 0
    got = out.stdout.strip("\n").split("\n")
    assert len(got) == 2 * len(want)
    for i, (cols, rows) in enumerate(want):
        assert np.array_equal(np.array(got[2 * i].split(), np.int64), cols), i
        assert np.array_equal(np.array(got[2 * i + 1].split(), np.int64), rows), i
