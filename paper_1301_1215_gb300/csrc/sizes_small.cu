#include "sizes.cuh"
namespace nlv {
const SizeKernels* sizes_small(int n) {
  switch (n) {
    NLV_SIZE_CASE(16, 4, 4)
    NLV_SIZE_CASE(32, 4, 8)
    NLV_SIZE_CASE(48, 4, 12)
    NLV_SIZE_CASE(64, 8, 8)
    NLV_SIZE_CASE(80, 4, 20)
    default: return nullptr;
  }
}
}  // namespace nlv
