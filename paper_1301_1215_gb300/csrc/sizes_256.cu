#include "sizes.cuh"
namespace nlv {
const SizeKernels* sizes_256(int n) {
  switch (n) {
    NLV_SIZE_CASE_TC(256, 16, 16)
    NLV_SIZE_CASE(320, 16, 20)
    default: return nullptr;
  }
}
}  // namespace nlv
