// Compiled variants of the sort for 64-bit key-value pairs.  Index 0 is the
// default multi-CTA shape; the others are candidates for the autotuner.
#include "rs_launch.cuh"

namespace rs {

const Variant* variants_kv64(int* count) {
  static const Variant table[] = {
      OnesweepSort<uint64_t, 8, 8, 256, 12, 2>::describe(),
      SmallSort<uint64_t, 8, 8, 512, 16>::describe(),
      OnesweepSort<uint64_t, 8, 8, 256, 8, 3>::describe(),
      OnesweepSort<uint64_t, 8, 8, 256, 16, 2>::describe(),
      SmallSort<uint64_t, 8, 8, 256, 16>::describe(),
      OnesweepSort<uint64_t, 8, 8, 256, 12, 2, true>::describe(),
      FusedSort<uint64_t, 8, 8, 256, 12, 2>::describe(),
      ClusterSort<uint64_t, 8, 8, 512, 8, 8>::describe(),
      OnesweepSort<uint64_t, 8, 8, 256, 13, 2, false, 16>::describe(),
      OnesweepSort<uint64_t, 8, 8, 256, 11, 2, false, 16>::describe(),
      OnesweepSort<uint64_t, 8, 8, 256, 23, 2, true, 16>::describe(),
      OnesweepSort<uint64_t, 8, 8, 256, 19, 2, true, 16>::describe(),
  };
  *count = int(sizeof(table) / sizeof(table[0]));
  return table;
}

}  // namespace rs
