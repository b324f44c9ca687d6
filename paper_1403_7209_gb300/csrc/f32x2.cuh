// Packed pairs of FP32 values on Blackwell's paired FP32 instructions
// (add / sub / mul / fma .rn.f32x2: two IEEE single-precision operations,
// each correctly rounded, per issued instruction).  A pair is two floats;
// the 64-bit register pairs the instructions need are formed inside each
// asm block, so ptxas can keep the two halves in adjacent registers.
#pragma once
#include <cuda_runtime.h>

namespace op2b {

struct f2 {
  float x, y;
};

__host__ __device__ __forceinline__ f2 mk2(float x, float y) { return f2{x, y}; }
__host__ __device__ __forceinline__ f2 splat2(float x) { return f2{x, x}; }

__device__ __forceinline__ f2 add2(f2 a, f2 b) {
  f2 r;
  asm("{.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rd, ra, rb;\n\t"
      "mov.b64 {%0, %1}, rd;}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}

__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
  f2 r;
  asm("{.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\t"
      "mov.b64 {%0, %1}, rd;}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}

__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
  f2 r;
  asm("{.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "mul.rn.f32x2 rd, ra, rb;\n\t"
      "mov.b64 {%0, %1}, rd;}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}

// a * b + c, each half rounded once
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  f2 r;
  asm("{.reg .b64 ra, rb, rc, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "mov.b64 rc, {%6, %7};\n\t"
      "fma.rn.f32x2 rd, ra, rb, rc;\n\t"
      "mov.b64 {%0, %1}, rd;}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return r;
}

// Knuth's two-sum on both halves: hi + lo += x, the addition's rounding
// error kept in lo (s + err == hi + x exactly in each half)
__device__ __forceinline__ void two_sum_acc2(f2& hi, f2& lo, f2 x) {
  const f2 s = add2(hi, x);
  const f2 bb = sub2(s, hi);
  const f2 err = add2(sub2(hi, sub2(s, bb)), sub2(x, bb));
  hi = s;
  lo = add2(lo, err);
}

}  // namespace op2b
