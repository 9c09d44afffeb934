// Deflection angle chi(b, E) of the classical scattering integral for the
// Jager potential form (Sec. 3.4.1-3.4.4) and the pair updates built on it.
//
//   chi = pi - 2 b int_{r_min}^inf dr / (r^2 sqrt(F(r))),  F = 1 - b^2/r^2 - V(r)/E,
//   r_min = the largest root of F.
//
// Per pair (one thread):
//  1. bracket: scan F downward from max(b, sigma0) (sigma0: zero of V, above
//     which F > 0 for every b) on a geometric grid, fine where orbiting can
//     create several roots (E below 1.5 well depths), coarse otherwise;
//  2. FP32 safeguarded Newton inside the bracket, then FP64 Newton steps
//     (the turning-point refinement);
//  3. u = r_min/r, u = 1 - s^2 turns the integral into
//       I = int_0^1 2 s ds / sqrt(G(s)),  G = F0 + (b/r_min)^2 s^2 (1+u) - dV/E,
//     smooth in s; an n-point Gauss-Legendre rule in FP32 on the difference
//     from the free-particle integrand (whose integral is known exactly),
//     so chi = -2 (b/r_min) int 2s (1/sqrt(G) - 1/sqrt(G0)) ds.  dV = V(r) - V(r_min)
//     is assembled from per-term differences written with exact identities
//     (1 - u^k = s^2 (1 + u + ... + u^(k-1)), expm1) so that it keeps FP32
//     relative accuracy as r -> r_min.
#include <cmath>
#include <mutex>
#include <vector>

#include "internal.cuh"
#include "pair.cuh"

namespace dsmc {

constexpr int kMaxNodes = 128;

__device__ __forceinline__ float tc_rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// e^x in FP64 for |x| < 700, written from the mathematics (Cody and Waite's
// additive argument reduction, then the Taylor series): x = n ln 2 + r with
// n = rint(x / ln 2) and r = (x - n L_hi) - n L_lo, where L_hi is ln 2
// truncated to 16 bits (n L_hi exact) and L_lo = ln 2 - L_hi to FP64; |r| <=
// ln2/2, so the Taylor polynomial of e^r to r^12 truncates below 2e-16
// relative; 2^n enters through the exponent field.  Seventeen FP64
// operations, within a few ulp of a correctly rounded e^x.
struct Exp64 {
  double inv_ln2, ln2_hi, ln2_lo;
  double c[13];   // 1/k!
};

__host__ inline Exp64 make_exp64() {
  Exp64 e;
  e.inv_ln2 = 1.0 / 0.6931471805599453;
  e.ln2_hi = 0.693145751953125;   // ln 2 truncated to 16 significant bits (n L_hi exact)
  // ln 2 - L_hi from the decimal expansion of ln 2 (0.69314718055994530941723212145817656807...)
  e.ln2_lo = 1.4286068203094172321214581765680755e-06;
  double f = 1.0;
  for (int k = 0; k <= 12; ++k) { if (k) f *= k; e.c[k] = 1.0 / f; }
  return e;
}

__device__ __forceinline__ double exp64(const Exp64& E, double x) {
  const double magic = 6755399441055744.0;   // 1.5 2^52: adding it rounds to an integer
  const double t = fma(x, E.inv_ln2, magic);
  const double n = t - magic;
  const int ni = __double2loint(t);          // n, from the low word
  const double r = fma(-n, E.ln2_lo, fma(-n, E.ln2_hi, x));
  double p = E.c[12];
#pragma unroll
  for (int k = 11; k >= 0; --k) p = fma(p, r, E.c[k]);
  return __hiloint2double(__double2hiint(p) + (ni << 20), __double2loint(p));
}


struct PotDev {
  int kind;
  int n_nodes;
  // Jager form (FP64 copies for the refinement, FP32 for the rest)
  double A, a1, a2, am1, am2, beta, C[6], rc, At, at;
  float fA, fa1, fa2, fam1, fam2, fbeta, fC[6], frc, fAt, fat;
  double Dd[17];      // FP64 copy of D
  double Dp[16];      // (p + 1) D_{p+1}: P'(r) = -r^-2 sum_p Dp_p r^-p
  double Dpp[16];     // (p + 1)(p + 2) D_{p+1}: P''(r) = r^-3 sum_p Dpp_p r^-p
  double Cd[6];       // (6 + 2n) C_n
  double Cdd[6];      // (6 + 2n)(7 + 2n) C_n
  float fDp[16], fCd[6];   // FP32 copies of Dp and Cd (the refinement's derivative)
  float D[17];        // P(r) = sum_p D_p r^-p,  e^{-beta r} P(r) = sum_n C_2n r^-2n e^{-x} S_2n(x)
  float Dlo[17];      // D_p - D[p] (D as an FP32 pair)
  float Clo[6];       // C_2n - fC[n]
  Exp64 ex64;         // constants of the FP64 exponential of the refinement
  float sigma0;       // zero crossing of V (F > 0 above max(b, sigma0))
  float orbit_E;      // below this energy use the fine bracket scan
  double d_hs, kappa, p;
  float fkappa, fp;
  float mass_over_4k; // E/k_B = mass g^2 / (4 k_B)
  // Gauss-Legendre nodes: [0, n_nodes) for every energy, [kMaxNodes,
  // kMaxNodes + n_low) with more nodes below orbit_E, where near-orbiting
  // pairs make the integrand steep (n_low = min(4 n_nodes, kMaxNodes))
  int n_low;
  float s_node[2 * kMaxNodes], w_node[2 * kMaxNodes];
};

// ---------------------------------------------------------------- FP32 pairs
// A value as an unevaluated sum hi + lo of two FP32 numbers (about 44
// significant bits), for products that need more than FP32 but not the
// FP64 pipe (about 1/64 of the FP32 rate on GB300): the exact product of two
// FP32 numbers from one FMA (Dekker / Kahan's error-free transformation),
// the cross terms added in FP32, the sum renormalised.
struct F2 {
  float hi, lo;
};
__device__ __forceinline__ F2 f2_mul(F2 a, F2 b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const float s = p + e;
  return F2{s, e - (s - p)};
}
// the FP32 rounding of (a_hi + a_lo)(b_hi + b_lo)
__device__ __forceinline__ float f2_mul_round(float ah, float al, F2 b) {
  const float p = ah * b.hi;
  float e = fmaf(ah, b.hi, -p);
  e = fmaf(ah, b.lo, e);
  e = fmaf(al, b.hi, e);
  return p + e;
}

// ---------------------------------------------------------------- FP64 potential
// V and V' in FP64, with the damped dispersion expanded into
//   -sum_n C_2n r^-2n + e^{-beta r} P(r),   P(r) = sum_p D_p r^-p,
// (exact: f_2n(x) = 1 - e^-x sum_{k<=2n} x^k/k!), evaluated by Horner in 1/r:
// one reciprocal and no other division.  The two parts cancel to at most
// about two decimal digits for r above the core radius, which FP64 absorbs.
__host__ __device__ inline double V64(const PotDev& P, double r, double* dV, double* rep_out = nullptr,
                                      double* ex_out = nullptr) {
  if (P.kind == 2) {
    const double v = P.kappa * pow(r, -P.p);
    *dV = -P.p * v / r;
    return v;
  }
  const double ir = 1.0 / r;
  if (r < P.rc) {
    const double e = P.At * exp(-P.at * r) * ir;
    *dV = -e * (P.at + ir);
    return e;
  }
  const double ir2 = ir * ir;
  const double rep = P.A * exp(P.a1 * r + P.a2 * r * r + P.am1 * ir + P.am2 * ir2);
  const double drep = rep * (P.a1 + 2.0 * P.a2 * r - P.am1 * ir2 - 2.0 * P.am2 * ir2 * ir);
  double q = 0.0, dq = 0.0, pw = ir2 * ir2 * ir2;  // sum C r^-2n and its derivative
#pragma unroll
  for (int n = 0; n < 6; ++n) {
    q = fma(P.C[n], pw, q);
    dq = fma(P.Cd[n], pw, dq);
    pw *= ir2;
  }
  dq *= -ir;
  double Pr = P.Dd[16], dPr = P.Dp[15];
#pragma unroll
  for (int k = 15; k >= 0; --k) Pr = fma(Pr, ir, P.Dd[k]);
#pragma unroll
  for (int k = 14; k >= 0; --k) dPr = fma(dPr, ir, P.Dp[k]);
  dPr *= -ir2;                                     // P'(r) = -sum p D_p r^-(p+1)
  const double ex = exp(-P.beta * r);
  if (rep_out) *rep_out = rep;
  if (ex_out) *ex_out = ex;
  *dV = drep - dq + ex * (dPr - P.beta * Pr);
  return rep - q + ex * Pr;
}

// V in FP64 at r (ir = 1/r given), the same expansion as V64, for the
// Newton refinement of the turning point, and V' in FP32: the derivative
// only sets the Newton step, and a relative error d in it leaves d times
// the step (about 1e-7 of a step that is itself about 1e-7 r: below 1e-13 r,
// or a linear rather than quadratic rate if the derivative cancels).  *rep,
// *ex receive A e^{poly} and e^{-beta r}, *Pr the damping polynomial P(r)
// (Jager form), from which the quadrature's coefficients are carried to the
// root, *dPr P'(r) and *dpoly poly'(r) in FP32 for that carry.
__device__ __forceinline__ double V64n(const PotDev& P, double r, double ir, float* dV, double* rep_out,
                                       double* ex_out, double* Pr_out, float* dPr_out, float* dpoly_out) {
  const double ir2 = ir * ir;
  *dPr_out = 0.f;
  *dpoly_out = 0.f;
  if (P.kind == 2) {
    const double v = P.kappa * pow(r, -P.p);
    *dV = f64_to_f32(-P.p * v * ir);
    return v;
  }
  if (r < P.rc) {
    const double e = P.At * exp(-P.at * r) * ir;
    *dV = f64_to_f32(-e * (P.at + ir));
    return e;
  }
  const double rep = P.A * exp64(P.ex64, P.a1 * r + P.a2 * r * r + P.am1 * ir + P.am2 * ir2);
  double q = 0.0, pw = ir2 * ir2 * ir2;
#pragma unroll
  for (int n = 0; n < 6; ++n) {
    q = fma(P.C[n], pw, q);
    pw *= ir2;
  }
  double Pr = P.Dd[16];
#pragma unroll
  for (int k = 15; k >= 0; --k) Pr = fma(Pr, ir, P.Dd[k]);
  const double ex = exp64(P.ex64, -P.beta * r);
  // the derivative in FP32
  const float rf = f64_to_f32(r), irf = f64_to_f32(ir), ir2f = irf * irf;
  const float ppf = P.fa1 + 2.f * P.fa2 * rf - P.fam1 * ir2f - 2.f * P.fam2 * ir2f * irf;   // poly'
  float dqf = 0.f, pwf = ir2f * ir2f * ir2f;
#pragma unroll
  for (int n = 0; n < 6; ++n) {
    dqf = fmaf(P.fCd[n], pwf, dqf);
    pwf *= ir2f;
  }
  dqf *= -irf;
  float dPrf = P.fDp[15];
#pragma unroll
  for (int k = 14; k >= 0; --k) dPrf = fmaf(dPrf, irf, P.fDp[k]);
  dPrf *= -ir2f;                                   // P'(r) = -sum p D_p r^-(p+1)
  const float repf = f64_to_f32(rep), exf = f64_to_f32(ex), Prf = f64_to_f32(Pr);
  *rep_out = rep;
  *ex_out = ex;
  *Pr_out = Pr;
  *dPr_out = dPrf;
  *dpoly_out = ppf;
  *dV = repf * ppf - dqf + exf * (dPrf - P.fbeta * Prf);
  return rep - q + ex * Pr;
}

// 1/x in FP64 without a division: the FP32 reciprocal (relative error
// about 2^-23) refined by Newton's iteration r <- r (2 - x r), written
// r + r (1 - x r): each step squares the relative error (2^-46, then below
// FP64 rounding).  x positive and inside the FP32 normal range.
__device__ __forceinline__ double rcp64_1(double x) {
  const double r = f32_to_f64(tc_rcp(f64_to_f32(x)));
  return fma(r, fma(-x, r, 1.0), r);
}
__device__ __forceinline__ double rcp64(double x) {
  const double r = rcp64_1(x);
  return fma(r, fma(-x, r, 1.0), r);
}

// sqrt(x) for x in [0, 1]: y = x / sqrt(x) from the FP32 reciprocal square
// root, then one FP64 Newton step on y^2 = x (relative error about 2^-46,
// far below the FP32 rounding the impact parameter then takes).  x = 0 -> 0.
__device__ __forceinline__ double sqrt64(double x) {
  const float xf = f64_to_f32(x);
  if (!(xf > 0.f)) return 0.0;
  const double y = x * f32_to_f64(rsqrtf(xf));
  return fma(0.5 * (x - y * y), f32_to_f64(rsqrtf(xf)), y);
}

// ---------------------------------------------------------------- FP32 potential
// V = A e^{poly} - sum_n C_2n r^-2n + e^{-beta r} sum_p D_p r^-p  (r >= rc)
__device__ __forceinline__ float V32(const PotDev& P, float r, float* dV) {
  if (P.kind == 1) { *dV = 0.f; return 0.f; }
  if (P.kind == 2) {
    const float v = P.fkappa * __powf(r, -P.fp);
    *dV = -P.fp * v / r;
    return v;
  }
  const float ir = 1.f / r;
  if (r < P.frc) {
    const float e = P.fAt * __expf(-P.fat * r) * ir;
    *dV = -e * (P.fat + ir);
    return e;
  }
  const float rep = P.fA * __expf(P.fa1 * r + P.fa2 * r * r + P.fam1 * ir + P.fam2 * ir * ir);
  const float drep = rep * (P.fa1 + 2.f * P.fa2 * r - P.fam1 * ir * ir - 2.f * P.fam2 * ir * ir * ir);
  const float ir2 = ir * ir;
  float q = 0.f, dq = 0.f, pw = ir2 * ir2 * ir2;
#pragma unroll
  for (int n = 0; n < 6; ++n) {
    q += P.fC[n] * pw;
    dq -= (6 + 2 * n) * P.fC[n] * pw * ir;
    pw *= ir2;
  }
  float Pr = P.D[16], dPr = 0.f;
#pragma unroll
  for (int p = 15; p >= 0; --p) {  // Horner in 1/r
    dPr = dPr * ir + (p + 1) * P.D[p + 1];
    Pr = Pr * ir + P.D[p];
  }
  dPr = -dPr * ir2;
  const float eb = __expf(-P.fbeta * r);
  *dV = drep - dq + eb * (dPr - P.fbeta * Pr);
  return rep - q + eb * Pr;
}

__device__ __forceinline__ float F32(const PotDev& P, float b2, float E, float r, float* dF) {
  float dV;
  const float V = V32(P, r, &dV);
  const float ir2 = 1.f / (r * r);
  *dF = 2.f * b2 * ir2 / r - dV / E;
  return 1.f - b2 * ir2 - V / E;
}

// ---------------------------------------------------------------- turning point
// The FP64 turning point and what the quadrature's coefficients reuse from
// its last FP64 evaluation, carried to the returned point.
struct Turn {
  double r, ir;        // r_min and 1/r_min
  double rep, ex;      // A e^{poly(r_min)}, e^{-beta r_min} (Jager form)
  double Pr;           // damping polynomial P(r_min)
};

// r_min in FP64: FP32 bracket + safeguarded Newton, then FP64 Newton steps
// (the turning-point refinement).  From the FP32 root (relative error about
// 1e-7) one step leaves about 1e-14.  Newton converges quadratically, so
// after a step eps the error is about (F''/2F') eps^2, below 1e-9 r for
// eps <= 2e-5 r away from orbiting; only a larger step (the FP32 stage ended
// away from the root) is followed by another (each extra iteration costs
// the whole warp).  The repulsion,
// e^{-beta r} and P(r) of the last evaluation are carried to the returned
// point by their Taylor series in the last step (|dpoly|, |beta dr| <
// 1e-5): their truncation is below 1e-10 relative, and the quadrature uses
// them in FP32.
// kWarp: every lane of the warp calls this together (a lane with nothing to
// compute on harmless inputs); the lanes leave the FP32 stage at different
// times, and the warp is reconverged before the FP64 steps, which then run
// for all lanes as long as any lane still refines (GB300's FP64 pipe costs a
// warp instruction however few lanes are active).
template <bool kWarp>
__device__ Turn rmin_device(const PotDev& P, float b, float E) {
  Turn T = {};
  if (P.kind == 1) {   // the same kind for every lane
    T.r = (double)fmaxf(b, (float)P.d_hs);
    T.ir = rcp64(T.r);
    return T;
  }
  const float b2 = b * b;
  float dF;
  float r_hi;
  if (P.kind == 0) r_hi = fmaxf(b, P.sigma0) * 1.000001f;
  else r_hi = fmaxf(b, __powf(P.fkappa / E, 1.f / P.fp)) * 2.f;
  const float q = (P.kind == 0 && E < P.orbit_E) ? 0.995f : 0.9f;
  float r_lo = r_hi;
  bool found = false;
  for (int t = 0; t < 4000; ++t) {
    r_lo = r_hi * q;
    if (F32(P, b2, E, r_lo, &dF) < 0.f) { found = true; break; }
    r_hi = r_lo;
    if (r_hi < 1e-3f) break;
  }
  const float r_nf = r_hi;   // the result when no sign change was found
  if (!kWarp && !found) {
    T.r = (double)r_nf;
    T.ir = rcp64(T.r);
    return T;
  }
  // safeguarded Newton in [r_lo, r_hi], F(r_lo) < 0 <= F(r_hi).  Convergence
  // is tested before the bisection fallback: a step below FP32 resolution
  // ends the iteration even when it lands on a bracket end.
  float r = r_hi;
  for (int it = 0; it < 24 && found; ++it) {
    const float f = F32(P, b2, E, r, &dF);
    if (f == 0.f) break;
    if (f < 0.f) r_lo = r; else r_hi = r;
    float rn = r - f / dF;
    const bool inside = rn >= r_lo && rn <= r_hi;
    if (fabsf(rn - r) <= 4e-7f * r) { if (inside) r = rn; break; }
    r = inside ? rn : 0.5f * (r_lo + r_hi);
  }
  // FP64 Newton steps, kept inside the FP32 bracket widened by 1e-4 (FP32
  // rounding can misplace its ends slightly)
  double rd = f32_to_f64(r), ir = rcp64(rd);
  const double lo = f32_to_f64(r_lo) * (1.0 - 1e-4), hi = f32_to_f64(r_hi) * (1.0 + 1e-4);
  const double bd2 = f32_to_f64(b) * f32_to_f64(b), iEd = rcp64(f32_to_f64(E));
  const float iEf = 1.f / E;
  double rep0 = 0.0, ex0 = 0.0, Pr0 = 0.0, dpoly = 0.0, dr = 0.0;
  float dPr0 = 0.f;
  if (kWarp) __syncwarp();
  bool act = found;
  for (int it = 0; it < 6; ++it) {
    if (kWarp ? !__any_sync(0xffffffffu, act) : !act) break;
    float dV, ppf;
    const double ir2 = ir * ir;
    const double V = V64n(P, rd, ir, &dV, &rep0, &ex0, &Pr0, &dPr0, &ppf);
    const double f = 1.0 - bd2 * ir2 - V * iEd;
    // F'(r) in FP32 (see V64n)
    const float irf = f64_to_f32(ir);
    const float df = 2.f * b2 * irf * irf * irf - dV * iEf;
    const double step = -f * f32_to_f64(1.f / df);
    const double rn = rd + step;
    // 1/rn from 1/rd: with s = step/rd, 1/(rd + step) = (1/rd)(1 - s + s^2 - ...),
    // truncated after s^2 (|s| < 1e-4: error below 1e-12 relative, then one
    // Newton step on the result)
    const double sr = step * ir;
    double irn = fma(ir, fma(sr, sr, -sr), ir);
    irn = fma(irn, fma(-rn, irn, 1.0), irn);
    if (act) {
      if (!(rn >= lo && rn <= hi) || !(df != 0.0)) {
        dr = 0.0;
        act = false;
      } else {
        dr = step;
        dpoly = step * f32_to_f64(ppf);
        ir = irn;
        rd = rn;
        if (fabs(step) <= 2e-5 * rd) act = false;
      }
    }
  }
  if (!found) {
    T.r = (double)r_nf;
    T.ir = rcp64(T.r);
    return T;
  }
  T.r = rd;
  T.ir = ir;
  if (P.kind == 0 && rd >= P.rc) {
    if (fabs(dr) <= 1e-4 * rd) {
      const double eb = -P.beta * dr;
      T.rep = rep0 * (1.0 + dpoly * (1.0 + 0.5 * dpoly));
      T.ex = ex0 * (1.0 + eb * (1.0 + 0.5 * eb));
      T.Pr = fma(f32_to_f64(dPr0), dr, Pr0);
    } else {  // a long last step (not converged): evaluate at rd
      float dV, dPr, ppf;
      V64n(P, rd, ir, &dV, &T.rep, &T.ex, &T.Pr, &dPr, &ppf);
    }
  }
  return T;
}

// ---------------------------------------------------------------- chi
// kWarp: see rmin_device (every lane of the warp calls it together).
template <bool kWarp = false>
__device__ float chi_device(const PotDev& P, float b_in, float E) {
  if (!kWarp && !(b_in > 0.f)) return (float)DSMC_PI;
  const float b = b_in > 0.f ? b_in : 1.f;   // b = 0: head-on, chi = pi (set at the end)
  const Turn Tp = rmin_device<kWarp>(P, b, E);
  const double rd = Tp.r, ird = Tp.ir;
  const float r0 = f64_to_f32(rd);
  const float bt = f64_to_f32(f32_to_f64(b) * ird);
  const float bt2 = bt * bt;
  const float iE = 1.f / E;
  float F0 = 0.f;
  if (P.kind == 1) F0 = 1.f - bt2;
  // per-pair coefficients about the FP64 turning point (Jager form), so that
  // the integrand's F(r_min) = 0 holds to FP64 rather than to FP32 rounding
  float d[17], qn[6], Rep0 = 0.f, e0 = 0.f, P0 = 0.f, Vc0 = 0.f, powk = 0.f;
  const bool core = P.kind == 0 && r0 < P.frc;
  if (P.kind == 0 && !core) {
    // d_p = D_p r0^-p and the dispersion coefficients C_2n r0^-2n, each the
    // FP32 rounding of a product formed with about 44 bits: the powers of
    // 1/r0 as FP32 pairs (1/r0 split from its FP64 value), the coefficients
    // as FP32 pairs
    const float ih = f64_to_f32(ird);
    const F2 ir2 = F2{ih, f64_to_f32(ird - f32_to_f64(ih))};
    F2 pw = F2{1.f, 0.f};
#pragma unroll
    for (int p = 0; p <= 16; ++p) {
      d[p] = p == 0 ? P.D[0] : f2_mul_round(P.D[p], P.Dlo[p], pw);
      if (p >= 6 && (p & 1) == 0) qn[(p - 6) >> 1] = f2_mul_round(P.fC[(p - 6) >> 1], P.Clo[(p - 6) >> 1], pw);
      pw = p == 0 ? ir2 : f2_mul(pw, ir2);
    }
    P0 = f64_to_f32(Tp.Pr);   // P(r0), carried from the last FP64 evaluation
    Rep0 = f64_to_f32(Tp.rep);
    e0 = f64_to_f32(Tp.ex);
  } else if (P.kind == 2) {
    Vc0 = (float)(P.kappa * pow(rd, -P.p));
    powk = P.fp;
  }
  double V0d = 0.0;
  if (core) { double dd; V0d = V64(P, rd, &dd); }
  float I = 0.f;
  const bool low = P.kind == 0 && E < P.orbit_E;
  const int q0 = low ? kMaxNodes : 0, q1 = q0 + (low ? P.n_low : P.n_nodes);
  for (int q = q0; q < q1; ++q) {
    const float s = P.s_node[q];
    const float w = s * s;          // 1 - u, exact
    const float u = 1.f - w;
    const float dr = r0 * w / u;    // r - r0
    float dV = 0.f;
    if (P.kind == 0 && !core) {
      const float r = r0 + dr;
      // repulsion: Rep0 * expm1(poly(r) - poly(r0))
      const float dpoly = dr * (P.fa1 + P.fa2 * (r + r0) - P.fam1 / (r * r0) -
                                P.fam2 * (r + r0) / (r * r * r0 * r0));
      const float drep = Rep0 * expm1f(dpoly);
      // G_k = 1 + u + ... + u^(k-1), so r^-k - r0^-k = -r0^-k w G_k
      float Gk = 0.f, uk = 1.f, dQ = 0.f, dP = 0.f;
#pragma unroll
      for (int k = 1; k <= 16; ++k) {
        Gk += uk;
        uk *= u;
        dP += d[k] * Gk;
        if ((k & 1) == 0 && k >= 6) dQ += qn[(k - 6) >> 1] * Gk;
      }
      dQ *= -w;                     // sum_n C (r^-2n - r0^-2n)
      dP *= -w;                     // P(r) - P(r0)
      const float dh = e0 * (expm1f(-P.fbeta * dr) * (P0 + dP) + dP);
      dV = drep - dQ + dh;
    } else if (P.kind == 2) {
      dV = Vc0 * expm1f(powk * log1pf(-w));  // kappa (r^-p - r0^-p)
    } else if (core) {
      double dd;
      dV = (float)(V64(P, rd + (double)dr, &dd) - V0d);
    }
    // G = G0 - dG with G0 = (b/r_min)^2 s^2 (1+u) the free-particle integrand;
    // integrate 1/sqrt(G) - 1/sqrt(G0) (its integral of G0 alone is
    // pi/(2 b/r_min) exactly), written as dG/(sqrt(G G0)(sqrt G + sqrt G0))
    // so that weak deflections keep their relative accuracy.
    const float G0 = bt2 * w * (1.f + u);
    const float dG = dV * iE - F0;
    const float G = fmaxf(G0 - dG, 1e-30f);
    const float rG = rsqrtf(G), rG0 = rsqrtf(G0);
    I += P.w_node[q] * 2.f * s * (dG * rG * rG0 / (G * rG + G0 * rG0));
  }
  return b_in > 0.f ? -2.f * bt * I : (float)DSMC_PI;
}

// ---------------------------------------------------------------- host set-up
static void gauss_legendre01(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = cos(DSMC_PI * (i + 0.75) / (n + 0.5)), pp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p1 = 1.0, p2 = 0.0;
      for (int k = 1; k <= n; ++k) {
        const double p3 = p2;
        p2 = p1;
        p1 = ((2.0 * k - 1.0) * z * p2 - (k - 1.0) * p3) / k;
      }
      pp = n * (z * p1 - p2) / (z * z - 1.0);
      const double dz = p1 / pp;
      z -= dz;
      if (fabs(dz) < 1e-15) break;
    }
    x[i] = 0.5 * (1.0 - z);
    w[i] = 1.0 / ((1.0 - z * z) * pp * pp);
  }
}

static PotDev make_pot(const dsmc_gas_t& gas, const dsmc_potential_t& p, int n_nodes) {
  PotDev P = {};
  P.kind = p.kind;
  P.n_nodes = n_nodes;
  P.A = p.A; P.a1 = p.a1; P.a2 = p.a2; P.am1 = p.am1; P.am2 = p.am2; P.beta = p.beta;
  for (int q = 0; q < 6; ++q) { P.C[q] = p.C[q]; P.fC[q] = (float)p.C[q]; }
  P.rc = 0.4 * p.R_eps; P.At = p.At; P.at = p.at;
  P.fA = (float)p.A; P.fa1 = (float)p.a1; P.fa2 = (float)p.a2; P.fam1 = (float)p.am1;
  P.fam2 = (float)p.am2; P.fbeta = (float)p.beta; P.frc = (float)P.rc; P.fAt = (float)p.At;
  P.fat = (float)p.at;
  P.d_hs = p.d_hs; P.kappa = p.kappa; P.p = p.p; P.fkappa = (float)p.kappa; P.fp = (float)p.p;
  P.mass_over_4k = (float)(gas.mass / (4.0 * DSMC_KB));
  P.ex64 = make_exp64();
  // D_p = sum_{n: 2n >= p} C_2n beta^(2n-p) / (2n-p)!
  for (int pp = 0; pp <= 16; ++pp) {
    double s = 0.0;
    for (int n = 3; n <= 8; ++n) {
      const int j = 2 * n - pp;
      if (j < 0) continue;
      double t = 1.0;
      for (int i = 1; i <= j; ++i) t *= p.beta / i;
      s += p.C[n - 3] * t;
    }
    P.D[pp] = (float)s;
    P.Dlo[pp] = (float)(s - (double)P.D[pp]);
    P.Dd[pp] = s;
  }
  for (int pp = 0; pp < 16; ++pp) P.Dp[pp] = (pp + 1) * P.Dd[pp + 1];
  for (int pp = 0; pp < 16; ++pp) P.Dpp[pp] = (double)(pp + 1) * (pp + 2) * P.Dd[pp + 1];
  for (int q = 0; q < 6; ++q) P.Cd[q] = (6 + 2 * q) * p.C[q];
  for (int pp = 0; pp < 16; ++pp) P.fDp[pp] = (float)P.Dp[pp];
  for (int q = 0; q < 6; ++q) P.fCd[q] = (float)P.Cd[q];
  for (int q = 0; q < 6; ++q) P.Clo[q] = (float)(p.C[q] - (double)P.fC[q]);
  for (int q = 0; q < 6; ++q) P.Cdd[q] = (double)(6 + 2 * q) * (7 + 2 * q) * p.C[q];
  if (p.kind == 0) {
    // sigma0: outermost zero of V (bisection on a sign change found inward from 4 R_eps)
    double dv, hi = 4.0 * p.R_eps, lo = hi;
    while (lo > 0.2 && V64(P, lo, &dv) < 0.0) lo *= 0.98;
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (V64(P, mid, &dv) < 0.0) hi = mid; else lo = mid;
    }
    P.sigma0 = (float)hi;
    double vmin = 0.0;
    for (double r = P.sigma0; r < 6.0 * p.R_eps; r *= 1.001) vmin = fmin(vmin, V64(P, r, &dv));
    P.orbit_E = (float)(1.5 * -vmin);
  }
  std::vector<double> x(n_nodes), w(n_nodes);
  gauss_legendre01(n_nodes, x.data(), w.data());
  for (int i = 0; i < n_nodes; ++i) { P.s_node[i] = (float)x[i]; P.w_node[i] = (float)w[i]; }
  P.n_low = 4 * n_nodes < kMaxNodes ? 4 * n_nodes : kMaxNodes;
  std::vector<double> xl(P.n_low), wl(P.n_low);
  gauss_legendre01(P.n_low, xl.data(), wl.data());
  for (int i = 0; i < P.n_low; ++i) { P.s_node[kMaxNodes + i] = (float)xl[i]; P.w_node[kMaxNodes + i] = (float)wl[i]; }
  return P;
}

// ---------------------------------------------------------------- kernels
// Warp-uniform loop: every lane of a warp computes chi together (a lane past
// the end, or with g = 0, on harmless inputs whose result is not kept).
__global__ void __launch_bounds__(128) k_jager_chi(PotDev P, int64_t n, const float* __restrict__ b,
                                                   const float* __restrict__ g, float* __restrict__ chi) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
    const int64_t q = base + lane;
    const bool valid = q < n;
    const float gg = valid ? g[q] : 0.f;
    const bool use = valid && gg > 0.f;
    const float c = chi_device<true>(P, use ? b[q] : 1.f, use ? P.mass_over_4k * gg * gg : 1.0e4f);
    if (valid) chi[q] = use ? c : 0.f;
  }
}

// cos and sin of an angle given in FP32: FP32 sincos, then the smaller of
// the two replaced by the FP64 square root of 1 - the larger squared, so
// that cos^2 + sin^2 = 1 to FP64 rounding (pair energy exact).
__device__ __forceinline__ void unit_angle(float ang, double* c, double* s) {
  float sf, cf;
  sincosf(ang, &sf, &cf);
  if (fabsf(cf) >= fabsf(sf)) {
    *s = (double)sf;
    *c = copysign(sqrt(1.0 - (double)sf * (double)sf), (double)cf);
  } else {
    *c = (double)cf;
    *s = copysign(sqrt(1.0 - (double)cf * (double)cf), (double)sf);
  }
}

// Deflect v_r = (u, v, w), |v_r| = g, 1/g = ig, by chi with azimuth eps
// (Bird 1994, Eq. 2.22), FP64; reciprocal square roots instead of divisions.
__device__ __forceinline__ void deflect(double u, double v, double w, double g, double ig, double cc,
                                        double sc, double ce, double se, double* o) {
  const double q2 = v * v + w * w;
  double cx, cy, cz, ax, ay, az;
  if (q2 > 0.0 && q2 > 1e-24 * (g * g)) {   // q > 1e-12 g
    const double iq = rsqrt(q2), q = q2 * iq, igq = iq * ig;
    cx = 0.0; cy = w * iq; cz = -v * iq;
    ax = q * ig; ay = -u * v * igq; az = -u * w * igq;
  } else {
    cx = 0.0; cy = 1.0; cz = 0.0;
    ax = 0.0; ay = 0.0; az = u >= 0.0 ? -1.0 : 1.0;
  }
  o[0] = cc * u + g * sc * (ce * cx + se * ax);
  o[1] = cc * v + g * sc * (ce * cy + se * ay);
  o[2] = cc * w + g * sc * (ce * cz + se * az);
}

struct JagerArgs {
  uint64_t seed, step;
  const uint64_t* step_dev;
  double bmax_A;
  const int4* pairs;
  const uint32_t* deps;
  const int32_t* ro;
  const dsmc_select_info_t* info;
  double *vx, *vy, *vz;
  float* chi_out;
  unsigned* done;
  unsigned* bar;   // [2] abort word, [3] unit cursor
  int* status;
};

// One pair: chi(b, E) for its impact parameter and energy, rotation of v_r
// (Bird 1994, Eq. 2.22) in FP64 -- cos and sin of the FP32 chi and of the
// azimuth eps = 2 pi U2 in FP64, so that the post-collision velocities are
// the exact deflection by that chi to FP64 rounding -- then the
// centre-of-mass update; velocities through L2.  Every lane of the warp runs
// it together (live false: a lane with no pair, or whose dependency wait
// failed, computes on harmless inputs and stores nothing), so that chi's FP64
// refinement and the FP64 rotation run with the warp converged.
__device__ __forceinline__ void collide_pair(const PotDev& P, const JagerArgs& a, int64_t p, int4 q, bool live) {
  double xi = 0.0, yi = 0.0, zi = 0.0, xj = 0.0, yj = 0.0, zj = 0.0;
  if (live) {
    xi = __ldcg(a.vx + q.x); yi = __ldcg(a.vy + q.x); zi = __ldcg(a.vz + q.x);
    xj = __ldcg(a.vx + q.y); yj = __ldcg(a.vy + q.y); zj = __ldcg(a.vz + q.y);
  }
  const double ux = xi - xj, uy = yi - yj, uz = zi - zj;
  const double g2 = ux * ux + uy * uy + uz * uz;
  const bool use = live && g2 > 0.0;
  const u32x4 w = draw(a.seed, (uint32_t)q.w, (uint32_t)q.z, a.step, TAG_JAGER);
  const float b = use ? f64_to_f32(a.bmax_A * sqrt64(u53_int(w.x, w.y))) : 1.f;
  const float E = use ? P.mass_over_4k * f64_to_f32(g2) : 1.0e4f;
  const float chi_c = chi_device<true>(P, b, E);
  const float chi = use ? chi_c : 0.f;
  if (live && a.chi_out) a.chi_out[p] = chi;
  __syncwarp();
  double sc, cc, se, ce;
  sincos(f32_to_f64(chi), &sc, &cc);
  sincospi(2.0 * u53_int(w.z, w.w), &se, &ce);
  const double g2s = use ? g2 : 1.0;
  const double ig = rsqrt(g2s);
  double o[3];
  deflect(use ? ux : 1.0, use ? uy : 0.0, use ? uz : 0.0, g2s * ig, ig, cc, sc, ce, se, o);
  if (!use) o[0] = o[1] = o[2] = 0.0;
  if (live) {
    const double cx = 0.5 * (xi + xj), cy = 0.5 * (yi + yj), cz = 0.5 * (zi + zj);
    __stcg(a.vx + q.x, cx + 0.5 * o[0]); __stcg(a.vy + q.x, cy + 0.5 * o[1]); __stcg(a.vz + q.x, cz + 0.5 * o[2]);
    __stcg(a.vx + q.y, cx - 0.5 * o[0]); __stcg(a.vy + q.y, cy - 0.5 * o[1]); __stcg(a.vz + q.y, cz - 0.5 * o[2]);
  }
}

// Pairs are claimed 32 at a time per warp, in round-major order, from one
// global cursor (units never span two rounds); each lane waits (bounded)
// until the previous pairs of its two particles are done, updates its pair
// and stamps both particles.  The cost of a pair varies by an order of
// magnitude (bracket scan, Newton iterations), so no warp waits for a round
// to end: only true dependencies order the work.  Which thread handles a
// pair does not change its result.
__global__ void __launch_bounds__(128, 4) k_collide_jager(PotDev P, JagerArgs a) {
  if (a.step_dev) a.step = *a.step_dev;
  const int R = a.info->n_rounds;
  const int lane = threadIdx.x & 31;
  int r = 0;
  int64_t base = 0;
  for (;;) {
    unsigned unit = 0;
    if (lane == 0) unit = atomicAdd(a.bar + 3, 1u);
    unit = __shfl_sync(0xffffffffu, unit, 0);
    int32_t p0, p1;
    if (!unit_range(a.ro, R, 32, r, base, unit, &p0, &p1)) break;
    const int32_t p = p0 + lane;
    const bool valid = p < p1;
    int4 q = make_int4(0, 0, 0, 0);
    bool ok = true;
    if (valid) {
      q = a.pairs[p];
      ok = wait_deps(a.done, q.x, q.y, a.deps[p], a.bar + 2, a.status);
    }
    __syncwarp();
    collide_pair(P, a, p, q, valid && ok);
    if (valid && ok) release_pair(a.done, q.x, q.y, (unsigned)(r + 1));
    if (!__all_sync(0xffffffffu, ok)) break;
  }
}

// ---------------------------------------------------------------- look-up table
// Sec. 3.4.4: the table of the look-up path over b~ = b/b_max (nb uniform
// nodes on [0, 1]) and E~ = ln(E_r/k_B) (nE uniform nodes on [lnE_min,
// lnE_max]), both ends included; filled here with the exact chi.
__global__ void __launch_bounds__(128) k_chi_table(PotDev P, int32_t nb, int32_t nE, double bmax_A, double lnE_min,
                                                   double dlnE, float* __restrict__ T) {
  const int64_t total = (int64_t)nb * nE;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = (int32_t)(q % nb), j = (int32_t)(q / nb);
    const float b = (float)(bmax_A * i / (nb - 1));
    const float E = (float)exp(lnE_min + j * dlnE);
    T[q] = chi_device(P, b, E);
  }
}

struct TableArgs {
  uint64_t seed, step;
  const uint64_t* step_dev;
  TableLook look;
  const int4* pairs;
  const uint32_t* deps;
  const int32_t* ro;
  const dsmc_select_info_t* info;
  double *vx, *vy, *vz;
  float* chi_out;
  unsigned* done;
  unsigned* bar;   // [2] abort word, [3] unit cursor
  int* status;
};

// The Jager pair update with chi from the table (b~ = sqrt(U1), eps = 2 pi U2
// from tag 4, E~ = ln(m g^2 / (4 k_B))); work claimed and ordered as in
// k_collide_jager.
__global__ void __launch_bounds__(256) k_collide_table(TableArgs a) {
  if (a.step_dev) a.step = *a.step_dev;
  const int R = a.info->n_rounds;
  const int lane = threadIdx.x & 31;
  int r = 0;
  int64_t base = 0;
  // a warp holds one unit (32 pairs of one round) and has already claimed the
  // next one, whose pair records load while the current pairs update; a unit
  // only ever waits on pairs claimed before it, so holding a later claim
  // cannot stall another warp
  auto claim = [&](int32_t* u0, int32_t* u1, int* ur) {
    unsigned unit = 0;
    if (lane == 0) unit = atomicAdd(a.bar + 3, 1u);
    unit = __shfl_sync(0xffffffffu, unit, 0);
    const bool got = unit_range(a.ro, R, 32, r, base, unit, u0, u1);
    *ur = r;
    return got;
  };
  int32_t p0 = 0, p1 = 0;
  int rc = 0;
  bool have = claim(&p0, &p1, &rc);
  int4 q = make_int4(0, 0, 0, 0);
  uint32_t dep = 0u;
  if (have && p0 + lane < p1) { q = a.pairs[p0 + lane]; dep = a.deps[p0 + lane]; }
  while (have) {
    int32_t n0 = 0, n1 = 0;
    int rn = 0;
    const bool next = claim(&n0, &n1, &rn);
    int4 qn = make_int4(0, 0, 0, 0);
    uint32_t depn = 0u;
    if (next && n0 + lane < n1) { qn = a.pairs[n0 + lane]; depn = a.deps[n0 + lane]; }
    const int32_t p = p0 + lane;
    const bool valid = p < p1;
    bool ok = true;
    if (valid) ok = wait_deps(a.done, q.x, q.y, dep, a.bar + 2, a.status);
    const bool live = valid && ok;
    double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (live) {
      v[0] = __ldcg(a.vx + q.x); v[1] = __ldcg(a.vy + q.x); v[2] = __ldcg(a.vz + q.x);
      v[3] = __ldcg(a.vx + q.y); v[4] = __ldcg(a.vy + q.y); v[5] = __ldcg(a.vz + q.y);
    }
    // every lane runs the pair update together after the warp reconverges
    // (as in k_collide_jager; a lane without a pair on zero velocities, its
    // result not stored)
    __syncwarp();
    const float chi = table_pair(a.look, a.seed, a.step, (uint32_t)q.w, (uint32_t)q.z, v);
    if (live) {
      if (a.chi_out) a.chi_out[p] = chi;
      __stcg(a.vx + q.x, v[0]); __stcg(a.vy + q.x, v[1]); __stcg(a.vz + q.x, v[2]);
      __stcg(a.vx + q.y, v[3]); __stcg(a.vy + q.y, v[4]); __stcg(a.vz + q.y, v[5]);
      release_pair(a.done, q.x, q.y, (unsigned)(rc + 1));
    }
    if (!__all_sync(0xffffffffu, ok)) break;
    have = next; p0 = n0; p1 = n1; rc = rn; q = qn; dep = depn;
  }
}

__global__ void __launch_bounds__(128) k_harvest(PotDev P, int64_t n, const double* __restrict__ vi,
                                                 const double* __restrict__ vj, const double* __restrict__ b,
                                                 const double* __restrict__ eps, double* __restrict__ vio,
                                                 double* __restrict__ vjo) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const double ux = vi[3 * p] - vj[3 * p], uy = vi[3 * p + 1] - vj[3 * p + 1], uz = vi[3 * p + 2] - vj[3 * p + 2];
    const double g2 = ux * ux + uy * uy + uz * uz;
    const float E = P.mass_over_4k * (float)g2;
    const float chi = g2 > 0.0 ? chi_device(P, (float)b[p], E) : 0.f;
    double cc, sc, ce, se;
    unit_angle(chi, &cc, &sc);
    unit_angle((float)eps[p], &ce, &se);
    double o[3] = {0.0, 0.0, 0.0};
    if (g2 > 0.0) {
      const double ig = rsqrt(g2);
      deflect(ux, uy, uz, g2 * ig, ig, cc, sc, ce, se, o);
    }
    for (int c = 0; c < 3; ++c) {
      const double cm = 0.5 * (vi[3 * p + c] + vj[3 * p + c]);
      vio[3 * p + c] = cm + 0.5 * o[c];
      vjo[3 * p + c] = cm - 0.5 * o[c];
    }
  }
}


// Self test of the refinement's FP64 helpers against CUDA's own routines:
// which 0: exp64, 1: exp, 2: rcp64, 3: 1.0 / x.
__global__ void k_selftest_math(Exp64 E, int which, int64_t n, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const double v = x[q];
    y[q] = which == 0 ? exp64(E, v) : which == 1 ? exp(v) : which == 2 ? rcp64(v) : 1.0 / v;
  }
}

static unsigned blocks_n(int64_t n, int threads, int cap) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}

int launch_selftest_math(Ctx* c, int which, int64_t n, const double* x, double* y, cudaStream_t s) {
  if (n == 0) return 0;
  k_selftest_math<<<blocks_n(n, 256, sm_count(c) * 8), 256, 0, s>>>(make_exp64(), which, n, x, y);
  count_launches(c, 1);
  return cudaGetLastError() == cudaSuccess ? 0 : DSMC_ERR_CUDA;
}

int launch_jager_chi(Ctx* c, const dsmc_gas_t& gas, const dsmc_potential_t& pot, int n_nodes,
                     int64_t n, const float* b, const float* g, float* chi, cudaStream_t s) {
  if (n == 0) return 0;
  const PotDev P = make_pot(gas, pot, n_nodes);
  const Shape sh = shape_or_default(c, DSMC_TUNE_JAGER_CHI);
  k_jager_chi<<<blocks_n(n, sh.threads, sm_count(c) * sh.blocks_per_sm), sh.threads, 0, s>>>(P, n, b, g, chi);
  count_launches(c, 1);
  return cudaGetLastError() == cudaSuccess ? 0 : DSMC_ERR_CUDA;
}

// resident blocks per SM of the Jager collide at a block size (0 on failure)
int occupancy_collide_jager(int threads) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k_collide_jager, threads, 0) != cudaSuccess)
    return 0;
  return per_sm;
}

int launch_collide_jager(Ctx* c, const dsmc_gas_t& gas, const dsmc_potential_t& pot,
                         int n_nodes, uint64_t step, int32_t n, const int32_t* pairs, const uint32_t* deps,
                         const int32_t* ro, const dsmc_select_info_t* info, double* vx, double* vy,
                         double* vz, float* chi_out, void* ws, size_t ws_bytes, cudaStream_t s) {
  if (ws_bytes < collide_ws(n)) return record(c, DSMC_ERR_ARG, "collide_jager: workspace too small");
  const Shape sh = shape_or_default(c, DSMC_TUNE_COLLIDE_JAGER);
  const int occ = occupancy_collide_jager(sh.threads);
  if (occ < 1) return record(c, DSMC_ERR_CUDA, "collide_jager: occupancy query failed");
  const int blocks = sm_count(c) * (sh.blocks_per_sm > 0 && sh.blocks_per_sm < occ ? sh.blocks_per_sm : occ);
  PotDev P = make_pot(gas, pot, n_nodes);
  JagerArgs a{gas.seed, step, graph_step_ptr(c), gas.b_max * 1e10, (const int4*)pairs, deps, ro, info, vx, vy, vz,
              chi_out, (unsigned*)ws, barrier_ptr(c), status_ptr(c)};
  if (cudaMemsetAsync(a.bar, 0, 4 * sizeof(unsigned), s) != cudaSuccess ||
      cudaMemsetAsync(a.done, 0, sizeof(unsigned) * (size_t)(n > 0 ? n : 1), s) != cudaSuccess)
    return DSMC_ERR_CUDA;
  k_collide_jager<<<blocks, sh.threads, 0, s>>>(P, a);
  count_launches(c, 1);
  return cudaGetLastError() == cudaSuccess ? 0 : record(c, DSMC_ERR_CUDA, "collide_jager: launch failed");
}

int launch_chi_table(Ctx* c, const dsmc_gas_t& gas, const dsmc_potential_t& pot, int n_nodes, int32_t nb,
                     int32_t nE, double lnE_min, double lnE_max, float* T, cudaStream_t s) {
  const PotDev P = make_pot(gas, pot, n_nodes);
  const int64_t total = (int64_t)nb * nE;
  k_chi_table<<<blocks_n(total, 128, sm_count(c) * 64), 128, 0, s>>>(P, nb, nE, gas.b_max * 1e10, lnE_min,
                                                                     (lnE_max - lnE_min) / (nE - 1), T);
  count_launches(c, 1);
  return cudaGetLastError() == cudaSuccess ? 0 : record(c, DSMC_ERR_CUDA, "chi_table: launch failed");
}

int occupancy_collide_table(int threads) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k_collide_table, threads, 0) != cudaSuccess)
    return 0;
  return per_sm;
}

int launch_collide_table(Ctx* c, const dsmc_gas_t& gas, const dsmc_chi_table_t& tab, uint64_t step, int32_t n,
                         const int32_t* pairs, const uint32_t* deps, const int32_t* ro,
                         const dsmc_select_info_t* info, double* vx, double* vy, double* vz, float* chi_out,
                         void* ws, size_t ws_bytes, cudaStream_t s) {
  if (ws_bytes < collide_ws(n)) return record(c, DSMC_ERR_ARG, "collide_table: workspace too small");
  const Shape sh = shape_or_default(c, DSMC_TUNE_COLLIDE_TABLE);
  const int occ = occupancy_collide_table(sh.threads);
  if (occ < 1) return record(c, DSMC_ERR_CUDA, "collide_table: occupancy query failed");
  const int blocks = sm_count(c) * (sh.blocks_per_sm > 0 && sh.blocks_per_sm < occ ? sh.blocks_per_sm : occ);
  TableArgs a;
  a.seed = gas.seed; a.step = step; a.step_dev = graph_step_ptr(c);
  a.look = table_look(gas, tab);
  a.pairs = (const int4*)pairs; a.deps = deps; a.ro = ro; a.info = info;
  a.vx = vx; a.vy = vy; a.vz = vz; a.chi_out = chi_out;
  a.done = (unsigned*)ws; a.bar = barrier_ptr(c); a.status = status_ptr(c);
  if (cudaMemsetAsync(a.bar, 0, 4 * sizeof(unsigned), s) != cudaSuccess ||
      cudaMemsetAsync(a.done, 0, sizeof(unsigned) * (size_t)(n > 0 ? n : 1), s) != cudaSuccess)
    return DSMC_ERR_CUDA;
  k_collide_table<<<blocks, sh.threads, 0, s>>>(a);
  count_launches(c, 1);
  return cudaGetLastError() == cudaSuccess ? 0 : record(c, DSMC_ERR_CUDA, "collide_table: launch failed");
}

int launch_harvest_jager(Ctx* c, const dsmc_gas_t& gas, const dsmc_potential_t& pot,
                         int n_nodes, int64_t n, const double* vi, const double* vj,
                         const double* b, const double* eps, double* vio, double* vjo,
                         cudaStream_t s) {
  if (n == 0) return 0;
  const PotDev P = make_pot(gas, pot, n_nodes);
  k_harvest<<<blocks_n(n, 128, sm_count(c) * 64), 128, 0, s>>>(P, n, vi, vj, b, eps, vio, vjo);
  count_launches(c, 1);
  return cudaGetLastError() == cudaSuccess ? 0 : DSMC_ERR_CUDA;
}

// ---------------------------------------------------------------- transport integrals
// Macroscopic validation (Eq. chapman_enskog and the two integrals after it;
// reading R8): Q2(E) = pi b_max^2 int_0^1 sin^2 chi(b_max sqrt(u), E) du by a
// composite 16-point Gauss-Legendre rule (b_panels equal panels of [0, 1]);
// Omega22(T) = 1/4 int_0^60 x^3 e^-x Q2(x T) dx by the same kind of rule
// (x_panels panels); mu = 5/16 sqrt(pi m k T) / Omega22.  One block per
// energy, chi at every node by the routine of the collide kernels, the
// block's sum in a fixed order (deterministic).
constexpr int kTrNodes = 16;
constexpr int kTrThreads = 256;
constexpr double kTrXmax = 60.0;

struct TransportArgs {
  int32_t n_e;
  const double* E;   // energies E_r/k_B (list mode), or null
  const double* T;   // temperatures (grid mode: energy e is x_j T_i, j = e % nx, i = e / nx)
  int32_t nx, x_panels, nb, b_panels;
  double bmax;
  double gl_x[kTrNodes], gl_w[kTrNodes];   // 16-point rule on [0, 1]
  double* q2;        // [n_e], m^2
  int* status;
};

__device__ __forceinline__ double tr_x(const TransportArgs& a, int32_t j) {
  return (j / kTrNodes + a.gl_x[j % kTrNodes]) * (kTrXmax / a.x_panels);
}

__global__ void __launch_bounds__(kTrThreads) k_transport_q2(PotDev P, TransportArgs a) {
  __shared__ double red[kTrThreads / 32];
  for (int32_t e = blockIdx.x; e < a.n_e; e += gridDim.x) {
    const double E = a.T ? tr_x(a, e % a.nx) * a.T[e / a.nx] : a.E[e];
    double acc = 0.0;
    if (E > 0.0 && E < 1e30) {   // chi takes E in FP32
      // the node's b only ever enters chi in FP32: formed in FP32 (GB300's
      // FP64 pipe bounds this kernel); the weights stay FP64
      const float inv_panels = 1.f / (float)a.b_panels, bmaxf = (float)a.bmax;
      for (int32_t k = threadIdx.x; k < a.nb; k += kTrThreads) {
        const int q = k % kTrNodes;
        const float u = ((float)(k / kTrNodes) + (float)a.gl_x[q]) * inv_panels;
        const float chi = chi_device(P, bmaxf * sqrtf(u), (float)E);
        const float sn = sinf(chi);
        acc += a.gl_w[q] * (double)(sn * sn);
      }
    } else if (threadIdx.x == 0) {
      set_status(a.status, DSMC_ERR_ARG);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double sum = 0.0;
      for (int w = 0; w < kTrThreads / 32; ++w) sum += red[w];
      a.q2[e] = DSMC_PI * a.bmax * a.bmax * (sum / a.b_panels) * 1e-20;
    }
    __syncthreads();
  }
}

// thread per temperature: Omega22 and mu from Q2 at the x nodes
__global__ void k_transport_finish(TransportArgs a, int32_t n_T, double mass, double* omega22, double* mu) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_T; i += gridDim.x * blockDim.x) {
    double om = 0.0;
    for (int32_t j = 0; j < a.nx; ++j) {
      const double x = tr_x(a, j);
      om += a.gl_w[j % kTrNodes] * (kTrXmax / a.x_panels) * x * x * x * exp(-x) * a.q2[(size_t)i * a.nx + j];
    }
    om *= 0.25;
    omega22[i] = om;
    mu[i] = 5.0 / 16.0 * sqrt(DSMC_PI * mass * DSMC_KB * a.T[i]) / om;
  }
}

static TransportArgs transport_args(Ctx* c, int32_t b_panels, double bmax) {
  TransportArgs a = {};
  std::vector<double> x(kTrNodes), w(kTrNodes);
  gauss_legendre01(kTrNodes, x.data(), w.data());
  for (int q = 0; q < kTrNodes; ++q) { a.gl_x[q] = x[q]; a.gl_w[q] = w[q]; }
  a.b_panels = b_panels;
  a.nb = b_panels * kTrNodes;
  a.bmax = bmax;
  a.status = status_ptr(c);
  return a;
}

size_t transport_ws(int32_t n_T, int32_t x_panels) {
  return align256(sizeof(double) * (size_t)(n_T > 0 ? n_T : 1) * kTrNodes * (size_t)x_panels);
}

int launch_transport_q2(Ctx* c, const dsmc_potential_t& pot, int n_nodes, int32_t n_E, const double* E,
                        double bmax, int32_t b_panels, double* q2, cudaStream_t s) {
  if (n_E == 0) return 0;
  dsmc_gas_t g = {};
  g.mass = 1.0;   // the mass enters only the energy of a velocity, unused here
  const PotDev P = make_pot(g, pot, n_nodes);
  TransportArgs a = transport_args(c, b_panels, bmax);
  a.n_e = n_E; a.E = E; a.q2 = q2;
  k_transport_q2<<<blocks_n(n_E, 1, sm_count(c) * 8), kTrThreads, 0, s>>>(P, a);
  count_launches(c, 1);
  return cudaGetLastError() == cudaSuccess ? 0 : DSMC_ERR_CUDA;
}

int launch_transport_viscosity(Ctx* c, const dsmc_gas_t& gas, const dsmc_potential_t& pot, int n_nodes,
                               int32_t n_T, const double* T, double bmax, int32_t b_panels, int32_t x_panels,
                               double* omega22, double* mu, void* ws, size_t ws_bytes, cudaStream_t s) {
  if (n_T == 0) return 0;
  if (ws_bytes < transport_ws(n_T, x_panels)) return record(c, DSMC_ERR_ARG, "transport: workspace too small");
  const PotDev P = make_pot(gas, pot, n_nodes);
  TransportArgs a = transport_args(c, b_panels, bmax);
  a.T = T; a.x_panels = x_panels; a.nx = x_panels * kTrNodes;
  a.n_e = n_T * a.nx;
  a.q2 = (double*)ws;
  k_transport_q2<<<blocks_n(a.n_e, 1, sm_count(c) * 8), kTrThreads, 0, s>>>(P, a);
  k_transport_finish<<<blocks_n(n_T, 128, sm_count(c)), 128, 0, s>>>(a, n_T, gas.mass, omega22, mu);
  count_launches(c, 2);
  return cudaGetLastError() == cudaSuccess ? 0 : DSMC_ERR_CUDA;
}

}  // namespace dsmc
