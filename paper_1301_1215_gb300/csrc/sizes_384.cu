#include "sizes.cuh"
namespace nlv {
const SizeKernels* sizes_384(int n) {
  switch (n) {
    NLV_SIZE_CASE(384, 16, 24)
    default: return nullptr;
  }
}
}  // namespace nlv
