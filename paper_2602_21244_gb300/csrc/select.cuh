// NTC selection (Sec. 2.2): the per-cell candidate count, the candidate
// draw, the screened accept decision and the round rule, shared by the
// selection kernels and the fused step.
#pragma once
#include <cmath>

#include "internal.cuh"

namespace dsmc {

struct SelArgs {
  const int32_t* cs;
  const double *vx, *vy, *vz;
  double* sgmax;
  double* sgnew;
  int32_t* counts;
  const int32_t* offs;
  int4* tmp;
  int32_t* tmp_round;
  uint32_t* tmp_dep;   // rounds (1-based, 0 = none) of the previous pair of i | of j << 16
  int32_t* wcnt;       // per cell: 32-candidate words of accept bits (ceil(M/32))
  int32_t* ncand;      // per cell: the NTC candidate count M (k_sel_nwords)
  const int32_t* wofs; // their exclusive scan (first word of each cell; [n_cells] = total)
  uint32_t* bits;      // accept bit of candidate m of cell k: bits[wofs[k] + m/32] >> (m % 32)
  int64_t words_cap;   // capacity of bits; a cell whose words do not fit is re-evaluated
  int32_t* last;
  int32_t* round_count;
  int32_t* n_rounds;
  unsigned long long* n_cand;
  int* status;
  int32_t n_cells;
  int32_t model;
  int64_t capacity;
  uint64_t seed, step;
  PhiloxKey key;             // round keys of seed
  const uint64_t* step_dev;  // if set, the step index is read here (graph replay)
  double fn, dt;
  // model 0: sigma(g) = pid2 * pow(x, om_half) / gam, x = two_kt / ((mr g) g)
  double pid2, om_half, gam, two_kt, mr;
  // model 1: sigma = sig_const
  double sig_const;
  // FP32 screen: sigma(g) g = k32 * g^e32 (e32 = 1 for model 1)
  float k32, e32;
  // bucket order of the pair list: 0 = rounds; 1 = claim levels, level =
  // round + (R - 1 - the last round of the pair's cell), R = the step's
  // round count (the emit pass then keeps each cell's last round in bits
  // 16.. of tmp_round)
  int32_t order;
};

__device__ __forceinline__ double sigma_g(const SelArgs& a, double g) {
  if (a.model == 1) return __dmul_rn(a.sig_const, g);
  const double x = __ddiv_rn(a.two_kt, __dmul_rn(__dmul_rn(a.mr, g), g));
  const double s = __ddiv_rn(__dmul_rn(a.pid2, pow(x, a.om_half)), a.gam);
  return __dmul_rn(s, g);
}

__device__ __forceinline__ int32_t ntc_count(const SelArgs& a, int32_t k, int32_t N, int* bad) {
  const u32x4 w = draw_k(a.key, 0, (uint32_t)k, a.step, TAG_NTC);
  double mt = __dmul_rn(0.5, (double)N);
  mt = __dmul_rn(mt, (double)(N - 1));
  mt = __dmul_rn(mt, a.fn);
  mt = __dmul_rn(mt, a.sgmax[k]);
  mt = __dmul_rn(mt, a.dt);
  const double mf = floor(__dadd_rn(mt, u53(w.x, w.y)));
  if (!(mf < 2147483647.0)) { *bad = 1; return 0; }
  return (int32_t)mf;
}

// A cell's FP64 velocities: particle i of the cell is vx[base + i] (any
// address space: the sorted arrays in global memory, or a shared-memory copy)
struct CellRef {
  const double *vx, *vy, *vz;
  int32_t base;
  __device__ __forceinline__ double x(uint32_t i) const { return vx[base + i]; }
  __device__ __forceinline__ double y(uint32_t i) const { return vy[base + i]; }
  __device__ __forceinline__ double z(uint32_t i) const { return vz[base + i]; }
};

// Exact FP64 decision for candidate pair (i, j) of cell k (the definition).
__device__ __forceinline__ bool decide64(const SelArgs& a, const CellRef& v, uint32_t i, uint32_t j,
                                         double U, double sgmax_k, double* sg_out) {
  const double dx = __dsub_rn(v.x(i), v.x(j));
  const double dy = __dsub_rn(v.y(i), v.y(j));
  const double dz = __dsub_rn(v.z(i), v.z(j));
  const double g2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  const double sg = sigma_g(a, __dsqrt_rn(g2));
  *sg_out = sg;
  return U < __ddiv_rn(sg, sgmax_k);
}

// Per-warp FP32 copy of a cell's velocities in shared memory (cells of up
// to kStage particles; larger cells read FP64 from global memory).
constexpr int kStage = 384;

struct CellView {
  const float *x, *y, *z;  // staged FP32 velocities, or null
  const float4* v4;        // or staged as (x, y, z, 0) per particle (one 16-byte load each)
  float dg;                // bound on the FP32 error of g for this cell
  float sgmax32, inv_sgmax32, thr_raise;
};

// Whether cell k's accept bits were kept: its word range lies inside the
// buffer and holds all M candidates (a range past the buffer, or a cell
// whose count was capped, is re-evaluated instead).
__device__ __forceinline__ bool bits_kept(const SelArgs& a, int32_t k, int32_t M) {
  const int64_t w0 = a.wofs[k], w1 = a.wofs[k + 1];
  return w0 >= 0 && w1 >= w0 && w1 <= a.words_cap && (w1 - w0) * 32 >= M;
}

// Particles (local indices) of candidate m of cell k (tag 2).
__device__ __forceinline__ void cand_ij(const SelArgs& a, int32_t k, int32_t N, int32_t m, int32_t* pi,
                                        int32_t* pj) {
  const u32x4 w = draw_k(a.key, (uint32_t)m, (uint32_t)k, a.step, TAG_CAND);
  const uint32_t i = mulhi_n(w.x, (uint32_t)N);
  uint32_t j = mulhi_n(w.y, (uint32_t)(N - 1));
  j += (j >= i);
  *pi = (int32_t)i; *pj = (int32_t)j;
}

// Candidate m of cell k.  The accept decision is screened in FP32 and taken
// in FP64 only when the FP32 ratio is within its error bound of U; the FP64
// sigma g is also formed for candidates that may raise (sigma g)_max.
// Returns accept; *raise_sg = FP64 sigma g if it may exceed the old maximum,
// else -1.
__device__ __forceinline__ bool candidate(const SelArgs& a, const CellView& cv, const CellRef& v, int32_t k,
                                          int32_t N, int32_t m, double sgmax_k, int32_t* pi, int32_t* pj,
                                          double* raise_sg) {
  const u32x4 w = draw_k(a.key, (uint32_t)m, (uint32_t)k, a.step, TAG_CAND);
  const uint32_t i = mulhi_n(w.x, (uint32_t)N);
  uint32_t j = mulhi_n(w.y, (uint32_t)(N - 1));
  j += (j >= i);
  *pi = (int32_t)i; *pj = (int32_t)j;
  float dx, dy, dz;
  if (cv.v4) {
    const float4 pi4 = cv.v4[i], pj4 = cv.v4[j];
    dx = pi4.x - pj4.x; dy = pi4.y - pj4.y; dz = pi4.z - pj4.z;
  } else if (cv.x) {
    dx = cv.x[i] - cv.x[j]; dy = cv.y[i] - cv.y[j]; dz = cv.z[i] - cv.z[j];
  } else {
    dx = (float)(v.x(i) - v.x(j));
    dy = (float)(v.y(i) - v.y(j));
    dz = (float)(v.z(i) - v.z(j));
  }
  // approximate square root and quotient (errors ~2^-22, far inside the
  // screen's 1e-4 relative margin; every decision near U is taken in FP64)
  float g;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(g) : "f"(dx * dx + dy * dy + dz * dz));
  const float sg = a.model == 1 ? a.k32 * g : a.k32 * __powf(g, a.e32);
  const float ratio = sg * cv.inv_sgmax32;
  // U32 <= U < U32 + 2^-24 (top 24 bits of the 53-bit uniform)
  const float U32 = (float)(w.z >> 8) * 5.9604645e-8f;
  // error bound of the FP32 ratio: 1e-4 relative (arithmetic, __powf) plus
  // the effect of the FP32 rounding of the velocities on g, ratio e32 dg/g;
  // for hard spheres (sigma g = k32 g, e32 = 1) that term is the cell's
  // constant k32 dg / (sigma g)_max, and dg/g > 1e-3 is g < 1e3 dg
  float margin;
  bool tiny_g;
  if (a.model == 1) {
    margin = 2e-7f + ratio * 1e-4f + a.k32 * cv.inv_sgmax32 * cv.dg;
    tiny_g = g < 1e3f * cv.dg;
  } else {
    const float relg = __fdividef(cv.dg, fmaxf(g, 1e-30f));
    margin = 2e-7f + ratio * (1e-4f + a.e32 * relg);
    tiny_g = relg > 1e-3f;
  }
  bool acc;
  double sg64 = -1.0;
  if (ratio > U32 + 5.9604645e-8f + margin) acc = true;
  else if (ratio < U32 - margin) acc = false;
  else acc = decide64(a, v, i, j, u53(w.z, w.w), sgmax_k, &sg64);
  if (sg > cv.thr_raise || tiny_g) {
    if (sg64 < 0.0) decide64(a, v, i, j, 0.0, sgmax_k, &sg64);
  } else {
    sg64 = -1.0;
  }
  *raise_sg = sg64;
  return acc;
}

// Rounds of a batch of up to 32 pairs taken in candidate order (lane order),
// by the rule round = 1 + max(round of the previous pair of i, of j).  Each
// active lane finds the nearest earlier lane of the batch touching each of
// its particles (per-particle lane masks), and the rounds follow from
// round = max(L_i, L_j), L = round + 1 of that lane, or the particle's round
// + 1 before the batch, by fixed-point iteration over shuffles: the links
// point to earlier lanes only, so it ends after (depth + 1) steps with the
// rounds of the sequential rule.  msk: one word per particle, zero on entry
// and on return; last: 1-based round of each particle's last pair (0 =
// none), updated.  Returns the 0-based round (clamped to DSMC_MAX_ROUNDS - 1,
// recording DSMC_ERR_UNSUPPORTED); *Li, *Lj = the 1-based rounds of the
// previous pairs of i and j (0 = none).  Called by the whole warp.
__device__ __forceinline__ int batch_rounds(bool act, uint32_t i, uint32_t j, uint32_t* msk, uint16_t* last,
                                            int* status, int* Li_out, int* Lj_out) {
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  if (act) { atomicOr(&msk[i], 1u << lane); atomicOr(&msk[j], 1u << lane); }
  __syncwarp();
  int pi = lane, pj = lane, lpi = 0, lpj = 0;
  bool lasti = false, lastj = false;
  if (act) {
    const uint32_t mi = msk[i], mj = msk[j];
    if (mi & below) pi = 31 - __clz(mi & below);
    if (mj & below) pj = 31 - __clz(mj & below);
    lasti = (mi >> lane) == 1u;   // no later lane of the batch touches i
    lastj = (mj >> lane) == 1u;
    lpi = last[i]; lpj = last[j];  // round + 1 before the batch (0 = none)
  }
  int r = max(lpi, lpj), Li = lpi, Lj = lpj;
  for (;;) {
    const int ri = __shfl_sync(0xffffffffu, r, pi), rj = __shfl_sync(0xffffffffu, r, pj);
    Li = pi == lane ? lpi : ri + 1;
    Lj = pj == lane ? lpj : rj + 1;
    const int rn = max(Li, Lj);
    const bool ch = act && rn != r;
    if (act) r = rn;
    if (!__any_sync(0xffffffffu, ch)) break;
  }
  __syncwarp();
  if (act) {
    if (r >= DSMC_MAX_ROUNDS) { set_status(status, DSMC_ERR_UNSUPPORTED); r = DSMC_MAX_ROUNDS - 1; }
    if (lasti) last[i] = (uint16_t)(r + 1);
    if (lastj) last[j] = (uint16_t)(r + 1);
    msk[i] = 0u; msk[j] = 0u;
  }
  __syncwarp();
  *Li_out = Li; *Lj_out = Lj;
  return r;
}

// The collision-model constants of SelArgs from the gas (host side).
inline void sel_model(SelArgs& a, const dsmc_gas_t& gas) {
  a.model = gas.model;
  a.pid2 = DSMC_PI * gas.d_ref * gas.d_ref;
  a.om_half = gas.omega - 0.5;
  a.gam = tgamma(2.5 - gas.omega);
  a.two_kt = 2.0 * DSMC_KB * gas.T_ref;
  a.mr = 0.5 * gas.mass;
  a.sig_const = DSMC_PI * gas.b_max * gas.b_max;
  if (gas.model == 1) { a.k32 = (float)a.sig_const; a.e32 = 1.f; }
  else {
    a.k32 = (float)(a.pid2 / a.gam * pow(a.two_kt / a.mr, a.om_half));
    a.e32 = (float)(2.0 - 2.0 * gas.omega);
  }
}

}  // namespace dsmc
