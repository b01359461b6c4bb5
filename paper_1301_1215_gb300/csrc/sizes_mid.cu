#include "sizes.cuh"
namespace nlv {
const SizeKernels* sizes_mid(int n) {
  switch (n) {
    NLV_SIZE_CASE(96, 8, 12)
    NLV_SIZE_CASE(128, 8, 16)
    NLV_SIZE_CASE(160, 8, 20)
    NLV_SIZE_CASE(192, 12, 16)
    default: return nullptr;
  }
}
}  // namespace nlv
