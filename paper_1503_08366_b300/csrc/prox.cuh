// Separable proximal operators (Section 5): base functions h and the parametric formula
//   prox_f(v) = (1/a) ( prox_{h, (e+rho)/(c a^2)} ( a (v rho - d)/(e + rho) - b ) + b ).
#pragma once
#include "common.cuh"

namespace pogs {

POGS_DEV float sigmoidf(float z) { return 1.0f / (1.0f + expf(-z)); }

// argmin_z log(1+e^z) + (r/2)(z - v)^2: the root of phi(z) = sigma(z) + r (z - v), which is
// strictly increasing, negative at v - 1/r and positive at v.  Safeguarded Newton: a step is
// replaced by bisection of the current bracket whenever it would leave the bracket or fails to
// halve the step before it (plain Newton can bounce between the two flat tails of the sigmoid
// without converging), so the bracket at least halves every other iteration.  The first guess
// is the root with sigma replaced by the piecewise-linear clamp(1/2 + z/4, 0, 1) (its middle
// piece, else the root of the tail's piece).  The iteration stops once |phi| is within the
// rounding error of its two terms (|phi| <= eps_32 (sigma + r |z - v|)): past that point a
// Newton step is noise, and at small r with large v (z far inside a wide bracket) the bisection
// fallback would otherwise halve the bracket down to the 1e-7 tolerance one step at a time.
POGS_DEV float prox_logistic(float v, float r) {
  float lo = v - 1.0f / r, hi = v;
  float z = (r * v - 0.5f) / (0.25f + r);
  if (z > 2.0f) z = fmaxf(lo, 2.0f);
  else if (z < -2.0f) z = fminf(v, -2.0f);
  z = fminf(fmaxf(z, lo), hi);
  float dx_old = hi - lo, dx = dx_old;
#pragma unroll 1
  for (int it = 0; it < 64; ++it) {
    const float s = sigmoidf(z);
    const float t = r * (z - v);
    const float phi = s + t;
    const float dphi = s * (1.0f - s) + r;
    if (fabsf(phi) <= 1.1920929e-7f * (s + fabsf(t))) break;
    if (phi > 0.0f) hi = z; else lo = z;
    const bool newton_out = ((z - hi) * dphi - phi) * ((z - lo) * dphi - phi) > 0.0f;
    const bool too_slow = fabsf(2.0f * phi) > fabsf(dx_old * dphi);
    dx_old = dx;
    if (newton_out || too_slow) {
      dx = 0.5f * (hi - lo);
      z = lo + dx;
    } else {
      dx = phi / dphi;
      z = z - dx;
    }
    if (fabsf(dx) <= 1e-7f * (1.0f + fabsf(z)) || hi - lo <= 1e-7f * (1.0f + fabsf(z))) break;
  }
  return z;
}

// argmin_{z > 0} z log z + (r/2)(z - v)^2: the root of psi(t) = t + 1 + r e^t - r v in
// t = log z.  psi is increasing and convex; with hi = max(v, 1) the root lies in
// [r (v - hi) - 1, log hi].  Newton from the right end (psi > 0) descends monotonically on a
// convex increasing function; as in the logistic prox, a step that leaves the bracket or
// fails to halve the previous one is replaced by bisection.
POGS_DEV float prox_xlogx(float v, float r) {
  const float zhi = fmaxf(v, 1.0f);
  float hi = logf(zhi), lo = r * (v - zhi) - 1.0f;
  float t = hi;
  float dx_old = hi - lo, dx = dx_old;
#pragma unroll 1
  for (int it = 0; it < 64; ++it) {
    const float et = expf(t);
    const float psi = t + 1.0f + r * et - r * v;
    const float dpsi = 1.0f + r * et;
    if (psi == 0.0f) break;
    if (psi > 0.0f) hi = t; else lo = t;
    const bool newton_out = ((t - hi) * dpsi - psi) * ((t - lo) * dpsi - psi) > 0.0f;
    const bool too_slow = fabsf(2.0f * psi) > fabsf(dx_old * dpsi);
    dx_old = dx;
    if (newton_out || too_slow) {
      dx = 0.5f * (hi - lo);
      t = lo + dx;
    } else {
      dx = psi / dpsi;
      t = t - dx;
    }
    if (fabsf(dx) <= 1e-7f * (1.0f + fabsf(t)) || hi - lo <= 1e-7f * (1.0f + fabsf(t))) break;
  }
  return expf(t);
}

// argmin_z h(z) + (r/2)(z - v)^2 for the base functions of the library.
POGS_DEV float prox_h(int h, float v, float r) {
  const float ir = 1.0f / r;
  switch (h) {
    case POGS_ZERO: return v;
    case POGS_ABS: return copysignf(fmaxf(fabsf(v) - ir, 0.0f), v);
    case POGS_SQUARE: return r * v / (1.0f + r);
    case POGS_HUBER: return fabsf(v) <= 1.0f + ir ? r * v / (1.0f + r) : v - copysignf(ir, v);
    case POGS_LOGISTIC: return prox_logistic(v, r);
    case POGS_HINGE: return v < 1.0f - ir ? v + ir : (v > 1.0f ? v : 1.0f);
    case POGS_MAXPOS: return v > ir ? v - ir : (v < 0.0f ? v : 0.0f);
    case POGS_IND_GE0: return fmaxf(v, 0.0f);
    case POGS_IND_LE0: return fminf(v, 0.0f);
    case POGS_IND_EQ0: return 0.0f;
    case POGS_IND_BOX01: return fminf(fmaxf(v, 0.0f), 1.0f);
    case POGS_XLOGX: return prox_xlogx(v, r);
    default: return v;
  }
}

// h(z) for the objective.  Indicators are evaluated as 0: the solver only evaluates f and g
// at prox outputs, which lie in the function's domain by construction.
POGS_DEV float h_value(int h, float z) {
  switch (h) {
    case POGS_ABS: return fabsf(z);
    case POGS_SQUARE: return 0.5f * z * z;
    case POGS_HUBER: return fabsf(z) <= 1.0f ? 0.5f * z * z : fabsf(z) - 0.5f;
    case POGS_LOGISTIC: return fmaxf(z, 0.0f) + log1pf(expf(-fabsf(z)));
    case POGS_HINGE: return fmaxf(0.0f, 1.0f - z);
    case POGS_MAXPOS: return fmaxf(0.0f, z);
    case POGS_XLOGX: return z > 0.0f ? z * logf(z) : 0.0f;
    default: return 0.0f;
  }
}

// Parametric prox of Section 5 at parameter rho.  c == 0 drops the h term (identity inner
// prox, the c -> 0 limit of the formula).
POGS_DEV float prox_param(int h, float a, float b, float c, float d, float e, float rho, float v) {
  const float w = a * (v * rho - d) / (e + rho) - b;
  const float z = c > 0.0f ? prox_h(h, w, (e + rho) / (c * a * a)) : w;
  return (z + b) / a;
}

POGS_DEV float f_param(int h, float a, float b, float c, float d, float e, float y) {
  const float hv = c > 0.0f ? c * h_value(h, a * y - b) : 0.0f;
  return hv + d * y + 0.5f * e * y * y;
}

}  // namespace pogs
