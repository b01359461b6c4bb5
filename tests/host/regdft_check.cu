// Host-side check of the register DFTs: every size used by the kernels, both directions, against the DFT
// sum evaluated in double.  Prints one line per size: "R D max_rel_err".
#include <cmath>
#include <cstdio>
#include <complex>
#include "fft_core.cuh"

template <int R, int D> double check() {
  float2 a[R];
  std::complex<double> ref[R], in[R];
  unsigned s = 12345u + R * 7 + (D > 0);
  for (int i = 0; i < R; ++i) {
    s = s * 1664525u + 1013904223u; float re = (s >> 8) / 16777216.0f - 0.5f;
    s = s * 1664525u + 1013904223u; float im = (s >> 8) / 16777216.0f - 0.5f;
    a[i] = make_float2(re, im);
    in[i] = {re, im};
  }
  for (int k = 0; k < R; ++k) {
    std::complex<double> acc = 0;
    for (int n = 0; n < R; ++n) acc += in[n] * std::polar(1.0, D * 2.0 * M_PI * n * k / R);
    ref[k] = acc;
  }
  nlv::RegDFT<R, D>::run(a);
  double num = 0, den = 0;
  for (int k = 0; k < R; ++k) {
    num += std::norm(std::complex<double>(a[k].x, a[k].y) - ref[k]);
    den += std::norm(ref[k]);
  }
  return std::sqrt(num / den);
}

template <int R> void both() {
  std::printf("%d -1 %.3e\n", R, check<R, -1>());
  std::printf("%d 1 %.3e\n", R, check<R, 1>());
}

int main() {
  both<2>(); both<3>(); both<4>(); both<5>(); both<6>(); both<8>(); both<10>(); both<12>(); both<15>();
  both<16>(); both<20>(); both<24>(); both<25>(); both<32>();
  std::printf("twiddle %.17g %.17g %.17g\n", nlv::unit_cos(1, 16), nlv::unit_sin(3, 24), nlv::unit_cos(7, 20));
  return 0;
}
