// Tuning variants of the sides 320, 384, 512 for nlinv_autotune: column strips of 4 and 16 columns for
// the default split, and the single-frame passes of an alternative four-step split.
#include "sizes.cuh"
namespace nlv {
int size_variants_b(int n, const SizeKernels** out, int max) {
  switch (n) {
    case 320: {
      static const ::nlv::SizeKernels s4 = ::nlv::make_size_kernels_strip<16, 20, 4>(*find_size(320));
      static const ::nlv::SizeKernels s16 = ::nlv::make_size_kernels_strip<16, 20, 16>(*find_size(320));
      int k = 0;
      if (k < max) out[k++] = find_size(320);
      if (k < max) out[k++] = &s4;
      if (k < max) out[k++] = &s16;
      static const ::nlv::SizeKernels alt = ::nlv::make_size_kernels_single<10, 32>();
      if (k < max) out[k++] = &alt;
      return k;
    }
    case 384: {
      static const ::nlv::SizeKernels s4 = ::nlv::make_size_kernels_strip<16, 24, 4>(*find_size(384));
      static const ::nlv::SizeKernels s16 = ::nlv::make_size_kernels_strip<16, 24, 16>(*find_size(384));
      int k = 0;
      if (k < max) out[k++] = find_size(384);
      if (k < max) out[k++] = &s4;
      if (k < max) out[k++] = &s16;
      static const ::nlv::SizeKernels alt = ::nlv::make_size_kernels_single<12, 32>();
      if (k < max) out[k++] = &alt;
      return k;
    }
    case 512: {
      static const ::nlv::SizeKernels s4 = ::nlv::make_size_kernels_strip<16, 32, 4>(*find_size(512));
      static const ::nlv::SizeKernels s16 = ::nlv::make_size_kernels_strip<16, 32, 16>(*find_size(512));
      int k = 0;
      if (k < max) out[k++] = find_size(512);
      if (k < max) out[k++] = &s4;
      if (k < max) out[k++] = &s16;
      return k;
    }
    default: return 0;
  }
}
}  // namespace nlv
