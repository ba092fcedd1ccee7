// Compiled variants of the sort for keys only, uint64_t keys.
#include "rs_launch.cuh"

namespace rs {

const Variant* variants_k64(int* count) {
  static const Variant table[] = {
      OnesweepSort<uint64_t, 0, 8, 256, 12, 3>::describe(),
      SmallSort<uint64_t, 0, 8, 512, 16>::describe(),
  };
  *count = int(sizeof(table) / sizeof(table[0]));
  return table;
}

}  // namespace rs
