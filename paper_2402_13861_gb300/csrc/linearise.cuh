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
//    - beta^2, a = erf(-mu / (sqrt 2 sigma)).  Evaluated as Phi = P(X > 0) and Q = 1 - Phi, both from
//  erfcf (so 1 - a^2 = 4 Phi Q has no cancellation), in units of sigma^2; gamma^2 is clamped at 0.
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
    float Phi = 0.5f * erfcf(-t * 0.70710678118654752f);
    float Q = 0.5f * erfcf(t * 0.70710678118654752f);
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

}  // namespace isx
