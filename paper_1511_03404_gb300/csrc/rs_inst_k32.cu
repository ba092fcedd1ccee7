// Compiled variants of the sort for 32-bit keys (keys only).  Index 0 is the
// default multi-CTA shape; the others are candidates for the autotuner
// (tile shape, registers per thread, digit width).
#include "rs_launch.cuh"

namespace rs {

const Variant* variants_k32(int* count) {
  static const Variant table[] = {
      OnesweepSort<uint32_t, 0, 8, 256, 16, 4>::describe(),
      SmallSort<uint32_t, 0, 8, 512, 16>::describe(),
      OnesweepSort<uint32_t, 0, 8, 256, 12, 4>::describe(),
      OnesweepSort<uint32_t, 0, 8, 256, 20, 3>::describe(),
      OnesweepSort<uint32_t, 0, 7, 256, 16, 4>::describe(),
      SmallSort<uint32_t, 0, 8, 256, 16>::describe(),
      OnesweepSort<uint32_t, 0, 8, 256, 16, 4, true>::describe(),
      OnesweepSort<uint32_t, 0, 8, 256, 16, 5>::describe(),
      FusedSort<uint32_t, 0, 8, 256, 16, 4>::describe(),
      FusedSort<uint32_t, 0, 8, 256, 8, 4>::describe(),
      ClusterSort<uint32_t, 0, 8, 512, 16, 8>::describe(),
      OnesweepSort<uint32_t, 0, 8, 256, 15, 4, true, 16>::describe(),
      OnesweepSort<uint32_t, 0, 8, 256, 17, 4, true, 16>::describe(),
      OnesweepSort<uint32_t, 0, 8, 256, 37, 2, true, 16, true>::describe(),
      OnesweepSort<uint32_t, 0, 8, 256, 37, 2, true, 16>::describe(),
      OnesweepSort<uint32_t, 0, 8, 256, 33, 2, true, 16>::describe(),
  };
  *count = int(sizeof(table) / sizeof(table[0]));
  return table;
}

}  // namespace rs
