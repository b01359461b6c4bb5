"""Host-side check of the launch geometry and shared-memory budgets of every compiled grid side.

The row-pass grid (nlv::row_grid), the column strips and the per-block shared memory of every pass are host
functions of kernels.cuh; this test compiles them into a small host program (nvcc, no device code instantiated) for
each grid side that sizes_*.cu compiles and checks, for 1..64 coils, fields of view 1, n/4 and n/2 and several SM
counts, that every coil row and image-plane pixel has a block, that a block's lanes fit its thread limit, and that
every pass -- single-frame, batched, standard-field-of-view and tensor-core forms -- fits the 227 KB of shared
memory a block may use on sm_103a.  No GPU is used."""
import os
import re
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1301_1215_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "kernels.cuh"
using namespace nlv;

template <int A, int B> SizeKernels table() {          // the geometry fields of make_size_kernels, no kernels
  SizeKernels s{};
  s.N1 = A; s.N2 = B;
  s.tl = Split<A, B>::TL;
  s.col_lanes = ColCfg<A, B>::C;
  s.col_threads = ColCfg<A, B>::THREADS;
  s.sm_lane = Split<A, B>::SM_LANE;
  s.sm_lane_col = Split<A, B>::SM_LANE_COL;
  return s;
}

struct Side { int n; bool tc; SizeKernels k; };
static const Side kSides[] = { SIDES };
constexpr size_t kSmemLimit = 227 * 1024 - 1024;   // dynamic shared memory per block, minus static use

static int bad = 0;
#define CHECK(c, ...) do { if (!(c)) { ++bad; std::printf("FAIL " __VA_ARGS__); std::printf("\n"); } } while (0)

int main() {
  int checked = 0;
  for (const Side& sd : kSides) {
    const SizeKernels& k = sd.k;
    const int N = sd.n;
    CHECK(k.N1 * k.N2 == N, "n=%d split %dx%d", N, k.N1, k.N2);
    const long plane = (long)N * N;
    for (int J = 1; J <= 64; ++J) {
      const int nrows = J * N;
      for (int sms : {1, 16, 152}) {
        for (int ctas : {1, 2, 3}) {
          for (long rho : {0L, plane}) {
            const RowGrid g = row_grid(&k, nrows, rho, sms, ctas);
            ++checked;
            CHECK(g.lanes >= 1 && g.lanes * k.tl <= kRowMaxThreads, "n=%d J=%d lanes %d", N, J, g.lanes);
            CHECK((long)g.blocks * g.rows_per_cta >= nrows, "n=%d J=%d rows not covered", N, J);
            CHECK((long)(g.blocks - 1) * g.rows_per_cta < nrows, "n=%d J=%d empty block", N, J);
            CHECK((long)g.rho_per_cta * g.blocks >= rho, "n=%d J=%d rho plane not covered", N, J);
            int lanes_tc = g.lanes;                 // tensor-core passes: whole warps
            while ((lanes_tc * k.tl) % 32 != 0) ++lanes_tc;
            for (int m = 0; m < NUM_ROW_MODES; ++m) {
              CHECK(k.row_smem(m, g.lanes) <= kSmemLimit, "n=%d J=%d row mode %d smem %zu", N, J, m,
                    k.row_smem(m, g.lanes));
              if (sd.tc) {
                CHECK(lanes_tc * k.tl <= kRowMaxThreads, "n=%d tc lanes %d", N, lanes_tc);
                CHECK(k.row_smem_tc(m, lanes_tc) <= kSmemLimit, "n=%d J=%d tc row mode %d smem %zu", N, J, m,
                      k.row_smem_tc(m, lanes_tc));
              }
            }
          }
        }
      }
      const int batch_lanes = kRowMaxThreads / k.tl;    // batch frames: fixed lanes
      for (int m = 0; m < NUM_ROW_MODES; ++m)
        CHECK(k.row_smem(m, batch_lanes) <= kSmemLimit, "n=%d batch row mode %d", N, m);
      for (int f : {1, N / 4, N / 2}) {
        const int Wc = 2 * f;
        const int strips = (Wc + k.col_lanes - 1) / k.col_lanes;
        CHECK(strips * k.col_lanes >= Wc && (strips - 1) * k.col_lanes < Wc, "n=%d f=%d strips", N, f);
        for (int m = 0; m < NUM_COL_MODES; ++m) {
          CHECK(k.col_smem(m, Wc) <= kSmemLimit, "n=%d f=%d col mode %d smem %zu", N, f, m, k.col_smem(m, Wc));
          if (sd.tc)
            CHECK(k.col_smem_tc(m, Wc) <= kSmemLimit, "n=%d f=%d tc col mode %d smem %zu", N, f, m,
                  k.col_smem_tc(m, Wc));
        }
      }
    }
  }
  std::printf("checked %d sides, %d grids, %d failures\n", (int)(sizeof(kSides) / sizeof(kSides[0])), checked, bad);
  return bad ? 1 : 0;
}
"""


def compiled_sides():
    sides = []
    for name in sorted(os.listdir(CSRC)):
        if name.startswith("sizes_") and name.endswith(".cu") and "tune" not in name:
            for tc, n, a, b in re.findall(r"NLV_SIZE_CASE(_TC)?\((\d+), (\d+), (\d+)\)", open(os.path.join(CSRC, name)).read()):
                sides.append((int(n), int(a), int(b), bool(tc)))
    return sorted(sides)


def test_compiled_sides_are_listed():
    sides = compiled_sides()
    assert {384, 512, 256, 128, 64} <= {n for n, *_ in sides}
    assert all(a * b == n for n, a, b, _ in sides)


def test_launch_geometry_and_shared_memory_of_every_side(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    table = ", ".join(f"{{{n}, {'true' if tc else 'false'}, table<{a}, {b}>()}}" for n, a, b, tc in compiled_sides())
    src = tmp_path / "geometry_check.cu"
    src.write_text(PROGRAM.replace("SIDES", table))
    exe = tmp_path / "geometry_check"
    r = subprocess.run([nvcc, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout[-3000:]
    assert "0 failures" in out.stdout
