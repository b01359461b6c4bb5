// Tuning variants of the sides 128, 192, 256 for nlinv_autotune: column strips of 4 and 16 columns for
// the default split, and the single-frame passes of an alternative four-step split.
#include "sizes.cuh"
namespace nlv {
int size_variants_a(int n, const SizeKernels** out, int max) {
  switch (n) {
    case 128: {
      static const ::nlv::SizeKernels s4 = ::nlv::make_size_kernels_strip<8, 16, 4>(*find_size(128));
      static const ::nlv::SizeKernels s16 = ::nlv::make_size_kernels_strip<8, 16, 16>(*find_size(128));
      int k = 0;
      if (k < max) out[k++] = find_size(128);
      if (k < max) out[k++] = &s4;
      if (k < max) out[k++] = &s16;
      static const ::nlv::SizeKernels alt = ::nlv::make_size_kernels_single<4, 32>();
      if (k < max) out[k++] = &alt;
      return k;
    }
    case 192: {
      static const ::nlv::SizeKernels s4 = ::nlv::make_size_kernels_strip<12, 16, 4>(*find_size(192));
      static const ::nlv::SizeKernels s16 = ::nlv::make_size_kernels_strip<12, 16, 16>(*find_size(192));
      int k = 0;
      if (k < max) out[k++] = find_size(192);
      if (k < max) out[k++] = &s4;
      if (k < max) out[k++] = &s16;
      static const ::nlv::SizeKernels alt = ::nlv::make_size_kernels_single<8, 24>();
      if (k < max) out[k++] = &alt;
      return k;
    }
    case 256: {
      static const ::nlv::SizeKernels s4 = ::nlv::make_size_kernels_strip<16, 16, 4>(*find_size(256));
      static const ::nlv::SizeKernels s16 = ::nlv::make_size_kernels_strip<16, 16, 16>(*find_size(256));
      int k = 0;
      if (k < max) out[k++] = find_size(256);
      if (k < max) out[k++] = &s4;
      if (k < max) out[k++] = &s16;
      static const ::nlv::SizeKernels alt = ::nlv::make_size_kernels_single<8, 32>();
      if (k < max) out[k++] = &alt;
      return k;
    }
    default: return 0;
  }
}
}  // namespace nlv
