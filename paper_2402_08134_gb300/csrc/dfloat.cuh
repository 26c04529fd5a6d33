// Double-float arithmetic: a value held as an unevaluated sum hi + lo of two
// floats, about 44-48 significant bits, on the FP32 pipes (GB300's FP64 rate
// is a small fraction of its FP32 rate).  Error-free transformations from
// Dekker (1971) and Knuth (TAOCP vol. 2): two-sum, fast two-sum (|a| >= |b|),
// and the product split by a fused multiply-add.
#pragma once

#include "common.cuh"

namespace symnmf {

struct dfl {
  float hi, lo;
};

SYMNMF_D dfl df_from_double(double v) {
  dfl r;
  r.hi = (float)v;
  r.lo = (float)(v - (double)r.hi);
  return r;
}
SYMNMF_D double df_to_double(dfl a) { return (double)a.hi + (double)a.lo; }

SYMNMF_D dfl df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return dfl{s, (a - (s - bb)) + (b - bb)};
}
SYMNMF_D dfl df_fast_two_sum(float a, float b) {
  const float s = a + b;
  return dfl{s, b - (s - a)};
}
SYMNMF_D dfl df_add(dfl a, dfl b) {
  dfl s = df_two_sum(a.hi, b.hi);
  s.lo += a.lo + b.lo;
  return df_fast_two_sum(s.hi, s.lo);
}
SYMNMF_D dfl df_mul(dfl a, dfl b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}
// c - a * b
SYMNMF_D dfl df_fms(dfl c, dfl a, dfl b) {
  const dfl p = df_mul(a, b);
  dfl s = df_two_sum(c.hi, -p.hi);
  s.lo += c.lo - p.lo;
  return df_fast_two_sum(s.hi, s.lo);
}
// 1 / sqrt(d) for d > 0: the FP32 estimate refined by one Newton step whose
// residual 1 - d y^2 is formed in double-float (relative error ~1e-13).
SYMNMF_D dfl df_rsqrt(dfl d) {
  const float y = rsqrtf(d.hi);
  const dfl ysq = df_mul(dfl{y, 0.f}, dfl{y, 0.f});
  const dfl r = df_fms(dfl{1.f, 0.f}, d, ysq);
  return df_fast_two_sum(y, 0.5f * y * (r.hi + r.lo));
}

}  // namespace symnmf
