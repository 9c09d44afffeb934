// Per-pair post-collision velocities of the CUDA-core update rules, shared
// by the collide kernels and the fused step: the VHS isotropic scatter
// (Sec. 2.1) and the deflection by a chi looked up in the table of the
// look-up path (Sec. 3.4.4), each with the centre-of-mass update (Sec. 2.3).
// A pair's random numbers are keyed by its candidate index m and cell k, so
// which thread runs a pair never changes its result.  Every rounding is
// explicit (the _rn intrinsics, fma): no multiply-add contraction is left to
// the compiler, so every kernel that inlines these functions computes the
// same bits.
#pragma once
#include "internal.cuh"

namespace dsmc {

// VHS (tag 3): v_r' = g (c, s cos e, s sin e), c = 2 U1 - 1, s = sqrt(1 - c^2),
// e = 2 pi U2; v = (vi, vj) in, post-collision (vi', vj') out.
__device__ __forceinline__ void vhs_pair(uint64_t seed, uint64_t step, uint32_t m, uint32_t k, double v[6]) {
  const double xi = v[0], yi = v[1], zi = v[2], xj = v[3], yj = v[4], zj = v[5];
  const double dx = __dsub_rn(xi, xj), dy = __dsub_rn(yi, yj), dz = __dsub_rn(zi, zj);
  const double g = sqrt(__fma_rn(dx, dx, __fma_rn(dy, dy, __dmul_rn(dz, dz))));
  const u32x4 w = draw(seed, m, k, step, TAG_ISO);
  const double c = __fma_rn(2.0, u53(w.x, w.y), -1.0);   // exact
  const double s = sqrt(__fma_rn(-c, c, 1.0));
  double se, ce;
  sincos(__dmul_rn(2.0 * DSMC_PI, u53(w.z, w.w)), &se, &ce);
  const double gs = __dmul_rn(g, s);
  const double rx = __dmul_rn(g, c), ry = __dmul_rn(gs, ce), rz = __dmul_rn(gs, se);
  const double cx = 0.5 * __dadd_rn(xi, xj), cy = 0.5 * __dadd_rn(yi, yj), cz = 0.5 * __dadd_rn(zi, zj);
  v[0] = __fma_rn(0.5, rx, cx); v[1] = __fma_rn(0.5, ry, cy); v[2] = __fma_rn(0.5, rz, cz);
  v[3] = __fma_rn(-0.5, rx, cx); v[4] = __fma_rn(-0.5, ry, cy); v[5] = __fma_rn(-0.5, rz, cz);
}

// The rotation of v_r = (ux, uy, uz) by chi with azimuth eps (Bird 1994,
// Eq. 2.22) with the direction in FP32 -- chi itself carries FP32 accuracy
// -- then scaled in FP64 to |v_r'| = |v_r| exactly: s = |v_r|/|y| from an
// FP32 estimate and one FP64 Newton step on s^2 |y|^2 = |v_r|^2 (relative
// error ~1e-14).  Returned as v_r' = 2 h Y (Y the FP32 rotated direction
// widened to FP64, h half the FP64 shell scale), so that a caller can form
// the post-collision velocities as c +- h Y with one FMA each.  The
// direction is within about 2e-6 rad of the exact deflection by the same
// chi and eps (the FP32 roundings of the inputs, the frame, sincosf and the
// FP32 azimuth); about a third of the FP64 work of an FP64 rotation.
__device__ __forceinline__ void deflect_shell_h(double ux, double uy, double uz, double g2, float chi, float eps,
                                                double* h, double* Yo) {
  const float fx = f64_to_f32(ux), fy = f64_to_f32(uy), fz = f64_to_f32(uz);
  float sc, cc, se, ce;
  sincosf(chi, &sc, &cc);
  sincosf(eps, &se, &ce);
  const float q2 = __fmaf_rn(fy, fy, __fmul_rn(fz, fz)), gf2 = __fmaf_rn(fx, fx, q2);
  const float gf = sqrtf(gf2);
  float cx, cy, cz, ax, ay, az;
  if (q2 > __fmul_rn(1e-24f, gf2) && q2 > 0.f) {
    const float iq = rsqrtf(q2), q = __fmul_rn(q2, iq), ig = __fdiv_rn(1.f, gf);
    const float iqg = __fmul_rn(iq, ig);
    cx = 0.f; cy = __fmul_rn(fz, iq); cz = __fmul_rn(-fy, iq);
    ax = __fmul_rn(q, ig); ay = __fmul_rn(__fmul_rn(-fx, fy), iqg); az = __fmul_rn(__fmul_rn(-fx, fz), iqg);
  } else {
    cx = 0.f; cy = 1.f; cz = 0.f;
    ax = 0.f; ay = 0.f; az = fx >= 0.f ? -1.f : 1.f;
  }
  const float gs = __fmul_rn(gf, sc);
  const float y0 = __fmaf_rn(cc, fx, __fmul_rn(gs, __fmaf_rn(ce, cx, __fmul_rn(se, ax))));
  const float y1 = __fmaf_rn(cc, fy, __fmul_rn(gs, __fmaf_rn(ce, cy, __fmul_rn(se, ay))));
  const float y2 = __fmaf_rn(cc, fz, __fmul_rn(gs, __fmaf_rn(ce, cz, __fmul_rn(se, az))));
  // the FP32 <-> FP64 conversions on the integer pipe (exact, and
  // correctly rounded to FP32): GB300's FP64 pipe, which runs the conversion
  // instructions, bounds this update
  const double Y0 = f32_to_f64(y0), Y1 = f32_to_f64(y1), Y2 = f32_to_f64(y2);
  Yo[0] = Y0; Yo[1] = Y1; Yo[2] = Y2;
  const double ny2 = __fma_rn(Y0, Y0, __fma_rn(Y1, Y1, __dmul_rn(Y2, Y2)));
  if (!(ny2 > 0.0)) { *h = 0.0; return; }
  const float ny2f = f64_to_f32(ny2), g2f = f64_to_f32(g2);
  // (|v_r|^2 below the FP32 normal range: v_r' = 0 up to ~1e-19 m/s)
  if (!(g2f > 0.f) || !(ny2f > 0.f)) { *h = 0.0; return; }
  const float sf = sqrtf(__fdiv_rn(g2f, ny2f));
  const double s0 = f32_to_f64(sf);
  const double res = __fma_rn(-__dmul_rn(s0, s0), ny2, g2);   // g2 - s0^2 ny2
  // one Newton step on s^2 ny2 = g2 from s0, halved: h = s / 2
  *h = __fma_rn(res, f32_to_f64(__fdiv_rn(__fmul_rn(0.25f, sf), g2f)), 0.5 * s0);
}

// The chi table of the look-up path in the form the pair update reads it.
struct TableLook {
  const float* T;
  int32_t nb, nE;
  float nb1;                 // nb - 1: x = b~ (nb - 1)
  float lnE_min, inv_dlnE;   // y = (ln E - lnE_min) inv_dlnE
  float mass_over_4k;
};

inline TableLook table_look(const dsmc_gas_t& gas, const dsmc_chi_table_t& tab) {
  TableLook L;
  L.T = tab.chi; L.nb = tab.nb; L.nE = tab.nE; L.nb1 = (float)(tab.nb - 1);
  L.lnE_min = (float)tab.lnE_min;
  L.inv_dlnE = (float)((tab.nE - 1) / (tab.lnE_max - tab.lnE_min));
  L.mass_over_4k = (float)(gas.mass / (4.0 * DSMC_KB));
  return L;
}

// chi by bilinear interpolation at (x, y) in node units, y clamped to the table
__device__ __forceinline__ float chi_lookup(const TableLook& a, float x, float y) {
  x = fminf(fmaxf(x, 0.f), (float)(a.nb - 1));
  y = fminf(fmaxf(y, 0.f), (float)(a.nE - 1));
  const int i0 = min((int)x, a.nb - 2), j0 = min((int)y, a.nE - 2);
  const float fx = __fsub_rn(x, (float)i0), fy = __fsub_rn(y, (float)j0);
  const float* r0 = a.T + (size_t)j0 * a.nb + i0;
  const float* r1 = r0 + a.nb;
  const float t00 = __ldg(r0), t01 = __ldg(r0 + 1), t10 = __ldg(r1), t11 = __ldg(r1 + 1);
  const float gx = __fsub_rn(1.f, fx);
  const float c0 = __fmaf_rn(fx, t01, __fmul_rn(gx, t00)), c1 = __fmaf_rn(fx, t11, __fmul_rn(gx, t10));
  return __fmaf_rn(fy, c1, __fmul_rn(__fsub_rn(1.f, fy), c0));
}

// The Jager pair update with chi from the table (tag 4: b~ = sqrt(U1),
// eps = 2 pi U2; E~ = ln(m g^2 / (4 k_B))); v in/out as in vhs_pair.
// Returns chi.
__device__ __forceinline__ float table_pair(const TableLook& L, uint64_t seed, uint64_t step, uint32_t m,
                                            uint32_t k, double v[6]) {
  const double xi = v[0], yi = v[1], zi = v[2], xj = v[3], yj = v[4], zj = v[5];
  const double ux = __dsub_rn(xi, xj), uy = __dsub_rn(yi, yj), uz = __dsub_rn(zi, zj);
  const double g2 = __fma_rn(ux, ux, __fma_rn(uy, uy, __dmul_rn(uz, uz)));
  const u32x4 w = draw(seed, m, k, step, TAG_JAGER);
  float chi = 0.f;
  double h = 0.0, Y[3] = {0.0, 0.0, 0.0};
  if (g2 > 0.0) {
    // the table coordinate and the azimuth only ever enter in FP32: their
    // uniforms are formed in FP32 too (GB300's FP64 pipe bounds this
    // update), to within one FP32 rounding of the FP64 values
    const float x = __fmul_rn(sqrtf(u_f32(w.x, w.y)), L.nb1);
    const float y = __fmul_rn(__fsub_rn(logf(__fmul_rn(L.mass_over_4k, f64_to_f32(g2))), L.lnE_min), L.inv_dlnE);
    chi = chi_lookup(L, x, y);
    deflect_shell_h(ux, uy, uz, g2, chi, __fmul_rn(u_f32(w.z, w.w), 6.2831855f), &h, Y);
  }
  const double sx = 0.5 * __dadd_rn(xi, xj), sy = 0.5 * __dadd_rn(yi, yj), sz = 0.5 * __dadd_rn(zi, zj);
  v[0] = fma(h, Y[0], sx); v[1] = fma(h, Y[1], sy); v[2] = fma(h, Y[2], sz);
  v[3] = fma(-h, Y[0], sx); v[4] = fma(-h, Y[1], sy); v[5] = fma(-h, Y[2], sz);
  return chi;
}

}  // namespace dsmc
