// Compiled variants of the sort for 64-bit keys (keys only).  Index 0 is the
// default multi-CTA shape; the others are candidates for the autotuner.
#include "rs_launch.cuh"

namespace rs {

const Variant* variants_k64(int* count) {
  static const Variant table[] = {
      OnesweepSort<uint64_t, 0, 8, 256, 12, 3>::describe(),
      SmallSort<uint64_t, 0, 8, 512, 16>::describe(),
      OnesweepSort<uint64_t, 0, 8, 256, 16, 3>::describe(),
      OnesweepSort<uint64_t, 0, 8, 256, 8, 4>::describe(),
      SmallSort<uint64_t, 0, 8, 256, 16>::describe(),
      OnesweepSort<uint64_t, 0, 8, 256, 12, 3, true>::describe(),
      FusedSort<uint64_t, 0, 8, 256, 12, 3>::describe(),
      ClusterSort<uint64_t, 0, 8, 512, 16, 8>::describe(),
      OnesweepSort<uint64_t, 0, 8, 256, 13, 3, true, 16>::describe(),
      OnesweepSort<uint64_t, 0, 8, 256, 11, 3, true, 16>::describe(),
      OnesweepSort<uint64_t, 0, 8, 256, 15, 3, true, 16, true>::describe(),
      OnesweepSort<uint64_t, 0, 8, 256, 27, 2, true, 16, true>::describe(),
      OnesweepSort<uint64_t, 0, 8, 256, 23, 2, true, 16>::describe(),
  };
  *count = int(sizeof(table) / sizeof(table[0]));
  return table;
}

}  // namespace rs
