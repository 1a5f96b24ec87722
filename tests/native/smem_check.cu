// Host-side check of the bulk kernel's shared-memory budget: the dynamic
// shared memory of each tile shape (StageSmem<R, TY>::bytes, a compile-time
// size) plus the kernel's static shared memory must let the resident blocks
// per SM the design counts on fit in the SM's 228 KB (each block also
// reserves 1 KB): two 16-row and four 8-row FP32 blocks (their launch bounds'
// 1024 threads), six 4-row FP32 blocks (768 threads: shared memory, not the
// launch bounds' eight, limits them), one FP64 block. Prints the sizes and
// exits non-zero if one does not fit.
#include <cstdio>

#include "m2c_stage.cuh"

template <typename R, int TY>
static int check(const char* name, int blocks_per_sm) {
  const size_t dyn = m2c::StageSmem<R, TY>::bytes;
  const size_t stat = sizeof(m2c::Grid) + 8 + 32 * 8 + 8 + 16;  // descriptor, dt, reduction, tile (upper bound)
  const size_t per_block = dyn + stat + 1024;
  const size_t sm = 228 * 1024;
  const bool ok = per_block * blocks_per_sm <= sm && dyn <= 227 * 1024;
  std::printf("%s: dynamic %zu B, per block %zu B, %d blocks/SM need %zu of %zu B: %s\n", name, dyn, per_block,
              blocks_per_sm, per_block * blocks_per_sm, sm, ok ? "fits" : "DOES NOT FIT");
  return ok ? 0 : 1;
}

int main() {
  int bad = 0;
  bad += check<float, 16>("FP32 16-row", 2);
  bad += check<float, 8>("FP32 8-row", 4);
  bad += check<float, 4>("FP32 4-row", 6);
  bad += check<double, 8>("FP64 8-row", 1);
  bad += check<double, 4>("FP64 4-row", 1);
  std::printf("misfits %d\n", bad);
  return bad == 0 ? 0 : 1;
}
