#include "sizes.cuh"
namespace nlv {
const SizeKernels* sizes_512(int n) {
  switch (n) {
    NLV_SIZE_CASE_TC(512, 16, 32)
    default: return nullptr;
  }
}
}  // namespace nlv
