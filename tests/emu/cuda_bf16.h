// cuda_bf16.h stand-in for the kernel emulation tests: the type and the one
// conversion the split path uses (small integers, exact in bfloat16).
#pragma once
#include <cstdint>
#include <cstring>
struct __nv_bfloat16 { uint16_t x; };
inline __nv_bfloat16 __float2bfloat16_rn(float f) {
  uint32_t b;
  memcpy(&b, &f, 4);
  b += 0x7fffu + ((b >> 16) & 1u);   // round to nearest even (exact for the small integers used)
  __nv_bfloat16 r;
  r.x = (uint16_t)(b >> 16);
  return r;
}
