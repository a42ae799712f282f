// Independent Philox4x32-10 for the oracle's pin: PyTorch's CPU engine
// (ATen/core/PhiloxRNGEngine.h).  Reads lines "c0 c1 c2 c3 k0 k1" and prints
// the four output words of the block at that counter under that key.
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdint>
#include <cstdio>

int main() {
  unsigned c[4], k[2];
  while (std::scanf("%u %u %u %u %u %u", &c[0], &c[1], &c[2], &c[3], &k[0], &k[1]) == 6) {
    // the engine's seed is the key, its offset words c0/c1, its subsequence c2/c3
    const uint64_t seed = (uint64_t)k[0] | ((uint64_t)k[1] << 32);
    const uint64_t sub = (uint64_t)c[2] | ((uint64_t)c[3] << 32);
    const uint64_t off = (uint64_t)c[0] | ((uint64_t)c[1] << 32);
    at::philox_engine e(seed, sub, off);
    const unsigned x0 = e(), x1 = e(), x2 = e(), x3 = e();
    std::printf("%u %u %u %u\n", x0, x1, x2, x3);
  }
  return 0;
}
