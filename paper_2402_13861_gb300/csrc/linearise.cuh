// Per-neuron ReLU linearisation shared by the float32 and tensor-core bound paths.
//
//  Sound affine arithmetic (Eq. 4, Chebyshev choice): the minimax line on [l, u].  For l < 0 < u it
//  is the chord through (l, 0) and (u, u) moved down by half its gap at 0:
//    alpha = u / (u - l),  beta = gamma = -alpha l / 2;   alpha = beta = gamma = 0 for u <= 0;
//    alpha = 1, beta = gamma = 0 for l >= 0.
//  With inflation the interval is widened by the slack delta, gamma is the exact maximum of
//  |relu(x) - alpha x - beta| over the three breakpoints l, 0, u (the error is piecewise linear),
//  rounded up, and alpha * delta plus the rounding of the new centre are added to gamma.
//
//  Uncertainty propagation (Eq. 9-10, Table VII, ReLU row) under N(mu, sigma^2):
//    alpha = (1 - a) / 2, beta = sigma phi(mu / sigma), gamma^2 = (1 - a^2)/4 (mu^2 + sigma^2) + a mu beta
//    - beta^2, a = erf(-mu / (sqrt 2 sigma)).  Evaluated as Phi = P(X > 0) and Q = 1 - Phi: the smaller
//  of the two from erfcf(|t| / sqrt 2) / 2 and the larger as its complement (so 1 - a^2 = 4 Phi Q has no
//  cancellation), in units of sigma^2; gamma^2 is clamped at 0.
//  sigma = 0 (or |mu| > 40 sigma): alpha = 1 if mu > 0, 1/2 if mu = 0, else 0; beta = gamma = 0.
#pragma once

#include <cuda_runtime.h>

namespace isx {

constexpr float kLinU = 5.9604645e-08f;   // 2^-24
constexpr float kLinSafe = 1.0000010f;    // 1 + 2^-20

struct Lin {
  float alpha, beta, gamma, center;
};

__device__ __forceinline__ Lin relu_clt(float mu, float sigma) {
  Lin r;
  if (sigma > 0.0f && fabsf(mu) < 40.0f * sigma) {
    float t = mu / sigma;
    // the smaller of Phi and Q from erfc of |t| (no cancellation), the other as its complement
    const float tail = 0.5f * erfcf(fabsf(t) * 0.70710678118654752f);
    const float Phi = t >= 0.0f ? 1.0f - tail : tail;
    const float Q = t >= 0.0f ? tail : 1.0f - tail;
    float phi = expf(-0.5f * t * t) * 0.39894228040143268f;
    r.alpha = Phi;
    r.beta = sigma * phi;
    float g2 = Phi * Q * (t * t + 1.0f) + (Q - Phi) * t * phi - phi * phi;
    r.gamma = sigma * sqrtf(fmaxf(g2, 0.0f));
  } else {
    r.alpha = mu > 0.0f ? 1.0f : (mu == 0.0f ? 0.5f : 0.0f);
    r.beta = 0.0f;
    r.gamma = 0.0f;
  }
  r.center = fmaf(r.alpha, mu, r.beta);
  return r;
}

// `rad` is the radius of the carried form, `delta` its slack (0 without inflation).
__device__ __forceinline__ Lin relu_sound(float c, float rad, float delta, bool inflate) {
  Lin r;
  float R = inflate ? __fadd_ru(__fmul_ru(rad, kLinSafe), delta) : rad;
  float l = inflate ? __fsub_rd(c, R) : c - R;
  float u = inflate ? __fadd_ru(c, R) : c + R;
  if (u <= 0.0f) {
    r.alpha = 0.0f; r.beta = 0.0f; r.gamma = 0.0f;
  } else if (l >= 0.0f) {
    r.alpha = 1.0f; r.beta = 0.0f; r.gamma = 0.0f;
  } else {
    r.alpha = u / (u - l);
    r.beta = -0.5f * r.alpha * l;
    if (inflate) {
      float e1 = fabsf(-r.alpha * l - r.beta), e2 = fabsf(r.beta), e3 = fabsf(u - r.alpha * u - r.beta);
      r.gamma = fmaxf(e1, fmaxf(e2, e3));
      r.gamma = __fadd_ru(r.gamma, 4.0f * kLinU * (fabsf(r.alpha * l) + fabsf(u) + fabsf(r.beta)));
    } else {
      r.gamma = r.beta;
    }
  }
  r.center = fmaf(r.alpha, c, r.beta);
  if (inflate) {
    r.gamma = __fadd_ru(r.gamma, __fmul_ru(r.alpha, delta));
    r.gamma = __fadd_ru(r.gamma, 2.0f * kLinU * (fabsf(r.alpha * c) + fabsf(r.beta)) * kLinSafe);
  }
  return r;
}

// ---- ELU and sine (least-squares rule only; the ISX_ACT_* codes) ----------------------------------
//
//  Both follow the definition of the least-squares line under X ~ N(mu, sigma^2):
//    alpha = Cov(f(X), X) / sigma^2,  beta = E f(X) - alpha mu,  gamma^2 = Var f(X) - alpha^2 sigma^2,
//  evaluated in forms whose float32 rounding error stays relative to the size of gamma^2 itself.
//
//  Sine (Table VII, sine row), s = sigma^2, a = e^{-s/2}:
//    alpha = a cos mu,  beta = a (sin mu - mu cos mu),
//    gamma^2 = P(s) + a^2 sin^2 mu q(s),  P(s) = (1 - e^{-2s}) / 2 - s e^{-s},  q(s) = s - (1 - e^{-s}),
//  which is Table VII's expression regrouped into two non-negative terms (both O(s^2) or smaller
//  for small s, where the printed form cancels O(s) terms).  For s < 1/2 both come from their
//  Taylor series, P = sum_{k>=3} (-1)^{k+1} (2^{k-1} - k) s^k / k!, q = sum_{k>=2} (-1)^k s^k / k!.
//
//  ELU, f = R + E with R = relu(X), E = (e^X - 1) [X <= 0] (so R E = 0), t = mu / sigma,
//  Phi = P(X > 0), Q = 1 - Phi, B1 = E[e^X; X <= 0], B2 = E[e^{2X}; X <= 0]:
//    alpha = Phi + B1,  beta = sigma phi(t) + B1 (1 - mu) - Q,
//    gamma^2 = gamma_R^2 + [Var E - sigma^2 B1^2] - 2 E[R] E[E] - 2 sigma^2 Phi B1,
//    Var E - sigma^2 B1^2 = B2 - (1 + sigma^2) B1^2 + Phi Q - 2 Phi B1,
//  gamma_R^2 the ReLU rule's residual variance.  B_s = exp(s mu + s^2 sigma^2 / 2) Phi(-(mu + s sigma^2)
//  / sigma) is taken as erfcx(y) e^{-t^2/2} / 2 for y = (t + s sigma) / sqrt 2 >= 0 (no overflow);
//  for y < 0 (mu < -s sigma^2) the bracket is written with e^{2 mu + sigma^2} factored out,
//  [e^{s2} - 1 - s2] - e2 e^{s2} + (2 e1 - e1^2)(1 + s2), s2 = sigma^2, e_s = erfc(-y_s) / 2, so
//  the lognormal part's O(sigma^4) residual is not a difference of O(1) terms.

namespace actmath {

constexpr float kInvSqrt2 = 0.70710678118654752f;
constexpr float kInvSqrt2Pi = 0.39894228040143268f;

// 1 / k! for k = 0 .. 13
__device__ __forceinline__ float inv_fact(int k) {
  constexpr float f[14] = {1.0f, 1.0f, 1.0f / 2, 1.0f / 6, 1.0f / 24, 1.0f / 120, 1.0f / 720, 1.0f / 5040,
                           1.0f / 40320, 1.0f / 362880, 1.0f / 3628800, 1.0f / 39916800, 1.0f / 479001600,
                           1.0f / 6227020800.0f};
  return f[k];
}

// P(s) = (1 - e^{-2s}) / 2 - s e^{-s} and q(s) = s - (1 - e^{-s}) for s >= 0.
__device__ __forceinline__ void sine_pq(float s, float& P, float& q) {
  if (s < 0.5f) {
    float p = 0.0f, c = 0.0f;
#pragma unroll
    for (int k = 13; k >= 3; --k) {
      const float ck = (float)((1 << (k - 1)) - k) * inv_fact(k);
      p = fmaf(p, s, (k & 1) ? ck : -ck);
    }
#pragma unroll
    for (int k = 12; k >= 2; --k) c = fmaf(c, -s, inv_fact(k));
    P = p * s * s * s;
    q = c * s * s;
  } else {
    P = fmaxf(-0.5f * expm1f(-2.0f * s) - s * expf(-s), 0.0f);
    q = fmaxf(s + expm1f(-s), 0.0f);
  }
}

// e^{s} - 1 - s for s >= 0.
__device__ __forceinline__ float expm1_minus(float s) {
  if (s < 0.5f) {
    float c = 0.0f;
#pragma unroll
    for (int k = 12; k >= 2; --k) c = fmaf(c, s, inv_fact(k));
    return c * s * s;
  }
  return expm1f(s) - s;
}

}  // namespace actmath

__device__ __forceinline__ Lin sine_clt(float mu, float sigma) {
  Lin r;
  float sn, cs;
  sincosf(mu, &sn, &cs);
  const float s = sigma * sigma;
  const float a = expf(-0.5f * s);
  r.alpha = a * cs;
  r.beta = a * (sn - mu * cs);
  float P, q;
  actmath::sine_pq(s, P, q);
  r.gamma = sqrtf(fmaxf(P + a * a * sn * sn * q, 0.0f));
  r.center = fmaf(r.alpha, mu, r.beta);
  return r;
}

__device__ __forceinline__ Lin elu_clt(float mu, float sigma) {
  Lin r;
  if (!(sigma > 0.0f)) {
    // the tangent at mu
    if (mu > 0.0f) {
      r.alpha = 1.0f;
      r.beta = 0.0f;
    } else {
      r.alpha = expf(mu);
      r.beta = expm1f(mu) - mu * r.alpha;
    }
    r.gamma = 0.0f;
    r.center = fmaf(r.alpha, mu, r.beta);
    return r;
  }
  const float t = mu / sigma;
  const float s2 = sigma * sigma;
  const float Phi = 0.5f * erfcf(-t * actmath::kInvSqrt2);
  const float Q = 0.5f * erfcf(t * actmath::kInvSqrt2);
  const float g = expf(-0.5f * t * t);
  const float phi = g * actmath::kInvSqrt2Pi;
  const float y1 = (t + sigma) * actmath::kInvSqrt2, y2 = (t + 2.0f * sigma) * actmath::kInvSqrt2;
  float B1, bracket;
  if (y2 >= 0.0f) {
    B1 = (y1 >= 0.0f) ? 0.5f * erfcxf(y1) * g : 0.5f * erfcf(y1) * expf(mu + 0.5f * s2);
    const float B2 = 0.5f * erfcxf(y2) * g;
    bracket = B2 - (1.0f + s2) * B1 * B1;
  } else {
    const float e1 = 0.5f * erfcf(-y1), e2 = 0.5f * erfcf(-y2);
    const float m = expf(mu + 0.5f * s2);
    B1 = (1.0f - e1) * m;
    const float es = expf(s2);
    bracket = m * m * (actmath::expm1_minus(s2) - e2 * es + (2.0f * e1 - e1 * e1) * (1.0f + s2));
  }
  const float ER = fmaf(mu, Phi, sigma * phi);
  const float EE = B1 - Q;
  const float g2R = s2 * (Phi * Q * (t * t + 1.0f) + (Q - Phi) * t * phi - phi * phi);
  const float g2 = g2R + bracket + Phi * Q - 2.0f * Phi * B1 - 2.0f * ER * EE - 2.0f * s2 * Phi * B1;
  r.alpha = Phi + B1;
  r.beta = sigma * phi + B1 * (1.0f - mu) - Q;
  r.gamma = sqrtf(fmaxf(g2, 0.0f));
  r.center = fmaf(r.alpha, mu, r.beta);
  return r;
}

// Least-squares rule of the INR's activation (ISX_ACT_RELU, ISX_ACT_ELU, ISX_ACT_SINE).
__device__ __forceinline__ Lin act_clt(int act, float mu, float sigma) {
  if (act == 1) return elu_clt(mu, sigma);
  if (act == 2) return sine_clt(mu, sigma);
  return relu_clt(mu, sigma);
}

// The activation itself.
__device__ __forceinline__ float act_fwd(int act, float z) {
  if (act == 1) return z > 0.0f ? z : expm1f(z);
  if (act == 2) return sinf(z);
  return fmaxf(z, 0.0f);
}

}  // namespace isx
