"""Host checks of the rasterizer's integer division helpers
(paper_2602_07782_gb300/csrc/raster_math.cuh compiled with g++): the
multiply-high division by the OBB table's divisors, the estimated 64-bit
floor division, the single-precision division by the OBB norms and the OBB
corner runs (started from one step's quotient, then advanced per
candidate) and the corner quantities at any scale equal exact floor
division.  The GPU parity tests check the
envelopes they produce against the oracle."""
from __future__ import annotations

import os
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <cstdio>
#include <cstdint>
#include <random>
#include "raster_math.cuh"
using namespace tabi::rmath;

static int64_t floor_div(int64_t a, int64_t d) {
  int64_t q = a / d;
  if ((a % d) != 0 && a < 0) --q;
  return q;
}

int main() {
  const uint32_t divisors[] = {16384, 16069, 15137, 13623, 11585, 9102, 6270, 3196, 2, 3, 7, 1000, 32767};
  std::mt19937_64 rng(12345);
  long bad = 0, checked = 0;
  const int32_t lim = 1 << 29;
  for (uint32_t d : divisors) {
    const Magic mg = magic_div(d);
    auto check = [&](int32_t a) {
      if (a <= -lim || a >= lim) return;
      ++checked;
      if (fdiv_magic(a, mg) != floor_div(a, d)) {
        if (bad < 5) std::printf("magic d=%u a=%d got %d want %lld\n", d, a, fdiv_magic(a, mg), (long long)floor_div(a, d));
        ++bad;
      }
    };
    for (int i = 0; i < 200000; ++i) check((int32_t)(rng() % (2u * lim)) - lim);
    // around multiples of d, across the whole range
    for (int64_t m = -(int64_t)lim / d - 1; m <= (int64_t)lim / d + 1; m += 1 + (int64_t)(lim / d) / 4096)
      for (int o = -2; o <= 2; ++o) check((int32_t)(m * (int64_t)d + o));
    for (int o = 0; o < 4096; ++o) { check(-lim + 1 + o); check(lim - 1 - o); check(o); check(-o); }
  }
  // 64-bit estimate: quotients below 2^40, numerators below 2^62
  for (int i = 0; i < 400000; ++i) {
    const int64_t d = (int64_t)(rng() % ((1ull << 46) - (1ull << 23))) + (1ll << 23);
    const int64_t a = (int64_t)(rng() % (1ull << 62)) - (1ll << 61);
    ++checked;
    if (fdiv64_est(a, d) != floor_div(a, d)) ++bad;
    const int64_t q = (int64_t)(rng() % (1ull << 38)) - (1ll << 37);
    for (int o = -1; o <= 1; ++o) {
      const int64_t b = q * d + o;
      if (b > -(1ll << 62) && b < (1ll << 62)) { ++checked; if (fdiv64_est(b, d) != floor_div(b, d)) ++bad; }
    }
  }
  // single-precision exact division by N in (2^23, 2^30), |a| < 2^62
  for (int i = 0; i < 400000; ++i) {
    const int64_t N = (int64_t)(rng() % ((1ull << 30) - (1ull << 23) - 1)) + (1ll << 23) + 1;
    const int64_t a = (int64_t)(rng() % (1ull << 63)) - (1ll << 62) + 1;
    ++checked;
    if (fdiv_n(a, N) != floor_div(a, N)) {
      if (bad < 5) std::printf("fdiv_n a=%lld N=%lld\n", (long long)a, (long long)N);
      ++bad;
    }
    const int64_t q = (int64_t)(rng() % (1ull << 39)) - (1ll << 38);
    for (int o = -2; o <= 2; ++o) {
      const int64_t b = q * N + o;
      if (b > -(1ll << 62) && b < (1ll << 62)) { ++checked; if (fdiv_n(b, N) != floor_div(b, N)) ++bad; }
    }
  }
  // OBB corner runs: a run started at candidate j0 from the per-chart step
  // (16 num = qs D + rs), then advanced one candidate at a time, gives
  // floor(k num / D) and its remainder at every k = 16 (j + 1)
  for (int t = 0; t < 3000; ++t) {
    int64_t C, S;
    do { C = (int64_t)(rng() % 16385); S = (int64_t)(rng() % 16385); } while (C * C + S * S <= (1ll << 23));
    auto r36 = [&]() { return (int64_t)(rng() % (1ull << 37)) - (1ll << 36); };
    const int64_t u0 = r36(), u1 = r36(), v0 = r36(), v1 = r36();
    const int item = (int)(rng() % 8);
    int64_t qs, rs;
    corner_step(item, C, S, u0, u1, v0, v1, qs, rs);
    const int64_t num = corner_num(item, C, S, u0, u1, v0, v1), D = corner_den(item, C, S);
    const int j0 = (int)(rng() % 64);
    CornerQ cq;
    corner_init(cq, item, j0, C, S, qs, rs);
    for (int j = j0; j < 64; ++j) {
      const int64_t kn = 16 * (int64_t)(j + 1) * num;
      const int64_t q = floor_div(kn, D);
      ++checked;
      if (cq.q != q || cq.r != kn - q * D) {
        if (bad < 5) std::printf("corner item %d j0 %d j %d got %lld want %lld\n", item, j0, j, (long long)cq.q, (long long)q);
        ++bad;
      }
      corner_advance(cq);
    }
  }
  // the same quantities at any scale k (the prefix-sum tail's trial and
  // intermediate scales): one division, floor(k num / D), and for the
  // positions whether it was exact
  for (int t = 0; t < 20000; ++t) {
    int64_t C, S;
    do { C = (int64_t)(rng() % 16385); S = (int64_t)(rng() % 16385); } while (C * C + S * S <= (1ll << 23));
    auto r36 = [&]() { return (int64_t)(rng() % (1ull << 37)) - (1ll << 36); };
    const int64_t u0 = r36(), u1 = r36(), v0 = r36(), v1 = r36();
    const int item = (int)(rng() % 8);
    const int64_t k = 1 + (int64_t)(rng() % 1024);
    const int64_t kn = k * corner_num(item, C, S, u0, u1, v0, v1), D = corner_den(item, C, S);
    CornerQ cq;
    corner_at(cq, item, k, C, S, u0, u1, v0, v1);
    const int64_t q = floor_div(kn, D);
    ++checked;
    if (cq.q != q || ((item & 3) >= 2 && (cq.r != 0) != (kn - q * D != 0))) {
      if (bad < 5) std::printf("corner_at item %d k %lld got %lld want %lld\n", item, (long long)k, (long long)cq.q, (long long)q);
      ++bad;
    }
  }
  std::printf("checked %ld bad %ld\n", checked, bad);
  return bad ? 1 : 0;
}
"""


def test_division_helpers_are_exact():
    gxx = "g++"
    with tempfile.TemporaryDirectory() as td:
        src = os.path.join(td, "t.cpp")
        exe = os.path.join(td, "t")
        with open(src, "w") as f:
            f.write(PROGRAM)
        inc = os.path.join(ROOT, "paper_2602_07782_gb300", "csrc")
        r = subprocess.run([gxx, "-O2", "-std=c++17", "-I", inc, src, "-o", exe], capture_output=True, text=True)
        if r.returncode != 0:
            pytest.fail(r.stderr[-3000:])
        r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stdout[-2000:]
        assert "bad 0" in r.stdout
