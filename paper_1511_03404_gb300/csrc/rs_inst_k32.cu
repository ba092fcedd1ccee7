// Compiled variants of the sort for keys only, uint32_t keys.
#include "rs_launch.cuh"

namespace rs {

const Variant* variants_k32(int* count) {
  static const Variant table[] = {
      OnesweepSort<uint32_t, 0, 8, 256, 16, 4>::describe(),
      SmallSort<uint32_t, 0, 8, 512, 16>::describe(),
  };
  *count = int(sizeof(table) / sizeof(table[0]));
  return table;
}

}  // namespace rs
