"""Host-side check of the tensor-core radix-16 stage's constant operand (tc_dft.cuh).

The B tiles (the real 32 x 32 form of the 16-point DFT matrix, split into bf16 hi and lo parts, forward and
inverse) are built on the host by nlv::host_tc_btables in the shared-memory tile layout.  This test compiles that
builder into a host program, reads the tiles back through the same layout function (tc_tile_offset), and evaluates
the three-pass split-BF16 contraction that the tensor cores perform -- A split as hi = bf16 truncation, lo = bf16
rounding of the remainder; hi*Bhi + hi*Blo + lo*Bhi accumulated -- in double for random vectors.  The result must
be the 16-point DFT of the vector to the split's precision (each operand keeps about 16 significant bits), and
exactly the DFT for the vectors the bf16 parts represent without rounding (a unit impulse).  No GPU is used."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1301_1215_gb300", "csrc")

PROGRAM = r"""
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include "tc_dft.cuh"
using namespace nlv;

static uint16_t trunc_bf16(float v) { uint32_t u; std::memcpy(&u, &v, 4); return (uint16_t)(u >> 16); }

int main() {
  static uint16_t tiles[kTcBBytes / 2];
  host_tc_btables(tiles);
  const double pi = 3.14159265358979323846;
  double worst = 0.0, rms_num = 0.0, rms_den = 0.0, impulse_err = 0.0;
  unsigned s = 2024u;
  for (int dir = 0; dir < 2; ++dir) {
    const double D = dir == 0 ? -1.0 : 1.0;
    const uint16_t* Bhi = tiles + (size_t)dir * 2 * (kTcBTileBytes / 2);
    const uint16_t* Blo = Bhi + kTcBTileBytes / 2;
    for (int trial = 0; trial < 201; ++trial) {
      float a[32];                                   // interleaved [Re x0, Im x0, Re x1, ...]
      for (int i = 0; i < 32; ++i) {
        s = s * 1664525u + 1013904223u;
        a[i] = (s >> 8) / 16777216.0f - 0.5f;
      }
      if (trial == 200) { for (int i = 0; i < 32; ++i) a[i] = 0.f; a[2 * 5] = 1.f; }   // impulse at n = 5
      double ahi[32], alo[32];
      for (int i = 0; i < 32; ++i) {
        ahi[i] = host_bf16_value(trunc_bf16(a[i]));
        alo[i] = host_bf16_value(host_bf16_rn((double)(a[i] - (float)ahi[i])));
      }
      for (int k = 0; k < 16; ++k) {
        double out[2];
        for (int b = 0; b < 2; ++b) {
          double acc = 0.0;
          for (int kk = 0; kk < 32; ++kk) {
            const int off = tc_tile_offset(2 * k + b, kk) / 2;
            const double bh = host_bf16_value(Bhi[off]), bl = host_bf16_value(Blo[off]);
            acc += ahi[kk] * bh + ahi[kk] * bl + alo[kk] * bh;
          }
          out[b] = acc;
        }
        std::complex<double> ref = 0.0;
        for (int n = 0; n < 16; ++n)
          ref += std::complex<double>(a[2 * n], a[2 * n + 1]) * std::polar(1.0, D * 2.0 * pi * n * k / 16.0);
        const double err = std::abs(std::complex<double>(out[0], out[1]) - ref);
        if (trial == 200) impulse_err = std::fmax(impulse_err, err);
        else {
          rms_num += err * err;
          rms_den += std::norm(ref);
          worst = std::fmax(worst, err);
        }
      }
    }
  }
  std::printf("%.3e %.3e %.3e\n", std::sqrt(rms_num / rms_den), worst, impulse_err);
  return 0;
}
"""


def test_tensor_core_b_tiles_give_the_16_point_dft(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "tc_tables.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "tc_tables"
    r = subprocess.run([nvcc, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    rel_rms, worst_abs, impulse = (float(v) for v in out)
    # a split keeps ~16 significant bits per operand: relative error of order 2^-16 (1.5e-5), far below bf16 alone
    assert rel_rms < 2e-5, rel_rms
    assert worst_abs < 1e-4, worst_abs
    # an impulse is represented exactly by its hi part; the output is a row of B, hi + lo of cos/sin: ~2^-17
    assert impulse < 1e-5, impulse
