// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC'11), written from the published round function:
// ten rounds of two 32x32->64 multiplications by 0xD2511F53 / 0xCD9E8D57 with
// the key bumped by the Weyl constants 0x9E3779B9 / 0xBB67AE85 between rounds.
#pragma once

#include <stdint.h>

namespace mochy {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// 64-bit uniform of draw n in `stream` (counter (n_lo, n_hi, stream, extra),
// key (seed_lo, seed_hi)): the first two output words, low word first.
__device__ __forceinline__ uint64_t philox_u64(uint64_t seed, uint64_t n, uint32_t stream,
                                               uint32_t extra) {
  const uint4 o = philox4x32_10(make_uint4((uint32_t)n, (uint32_t)(n >> 32), stream, extra),
                                (uint32_t)seed, (uint32_t)(seed >> 32));
  return ((uint64_t)o.y << 32) | o.x;
}

}  // namespace mochy
