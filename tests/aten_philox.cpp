// Test helper: ATen's own Philox4x32-10 engine (header-only, independent of
// this project's code), exported for a ctypes comparison against the oracle.
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdint>

extern "C" void aten_philox_block(uint64_t seed, uint64_t subsequence, uint64_t offset, uint32_t out[4]) {
    at::Philox4_32 eng(seed, subsequence, offset);
    for (int k = 0; k < 4; ++k) out[k] = eng();
}
