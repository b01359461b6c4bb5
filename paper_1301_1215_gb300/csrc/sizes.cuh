// Grid sides with compiled transforms and their four-step splits N = N1 * N2.  Each sizes_*.cu file instantiates
// the pass kernels of a few sides so that they compile in parallel.
#pragma once
#include "kernels.cuh"

namespace nlv {

// Lookup functions defined by the sizes_*.cu files: the kernel table of side n, or nullptr if that file does not
// hold n.
const SizeKernels* sizes_small(int n);
const SizeKernels* sizes_mid(int n);
const SizeKernels* sizes_256(int n);
const SizeKernels* sizes_384(int n);
const SizeKernels* sizes_512(int n);

// Tuning variants of side n (defined in sizes_tune_*.cu): up to max tables (the default first, then column strips
// of 4 and 16, then an alternative four-step split); returns their number (1 when n has no variants).
int size_variants_a(int n, const SizeKernels** out, int max);
int size_variants_b(int n, const SizeKernels** out, int max);
const SizeKernels* find_size(int n);
inline int size_variants(int n, const SizeKernels** out, int max) {
  int k = size_variants_a(n, out, max);
  if (k == 0) k = size_variants_b(n, out, max);
  if (k == 0 && max > 0 && find_size(n)) { out[0] = find_size(n); k = 1; }
  return k;
}

inline const SizeKernels* find_size(int n) {
  const SizeKernels* s = nullptr;
  if (!s) s = sizes_small(n);
  if (!s) s = sizes_mid(n);
  if (!s) s = sizes_256(n);
  if (!s) s = sizes_384(n);
  if (!s) s = sizes_512(n);
  return s;
}

}  // namespace nlv

#define NLV_SIZE_CASE(n, a, b)                                      \
  case n: {                                                         \
    static const ::nlv::SizeKernels k = ::nlv::make_size_kernels<a, b>(); \
    return &k;                                                      \
  }
// A side that also has the passes with tensor-core radix-16 stages.
#define NLV_SIZE_CASE_TC(n, a, b)                                   \
  case n: {                                                         \
    static const ::nlv::SizeKernels k = ::nlv::make_size_kernels_tc<a, b>(); \
    return &k;                                                      \
  }
