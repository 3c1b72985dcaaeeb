// Element types of the low-precision blocks: one complex number per element, either float2 or
// two BF16 numbers packed in a 32-bit word (re in the low half), with FP32 arithmetic on both.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace lp {

// Two BF16 numbers (re, im) in one 32-bit word, re in the low half.
struct bf16x2 {
  unsigned w;
};

// ------------------------------------------------------------------ element access
// A BF16 number is the upper half of the FP32 number with the same bits, so widening is a shift.
WD_DEV Cx<float> unpack(unsigned w) {
  return {__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u)};
}
WD_DEV unsigned pack(Cx<float> a) {   // round to nearest even
  const __nv_bfloat162 h = __floats2bfloat162_rn(a.re, a.im);
  return (unsigned)__bfloat16_as_ushort(h.x) | ((unsigned)__bfloat16_as_ushort(h.y) << 16);
}

WD_DEV Cx<float> ld1(const float2* p) {
  const float2 v = __ldg(p);
  return {v.x, v.y};
}
WD_DEV Cx<float> ld1(const bf16x2* p) { return unpack(__ldg(&p->w)); }

WD_DEV void st1(float2* p, Cx<float> a) { *p = make_float2(a.re, a.im); }
WD_DEV void st1(bf16x2* p, Cx<float> a) { p->w = pack(a); }

}  // namespace lp
