// cuda_bf16.h stand-in for the kernel emulation tests (the type only).
#pragma once
#include <cstdint>
struct __nv_bfloat16 { uint16_t x; };
