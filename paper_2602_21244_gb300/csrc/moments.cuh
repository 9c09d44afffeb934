// Exact integer cell moments (Sec. 2.5: the per-cell momentum and energy
// that moment matching restores), shared by the moment kernels and the fused step.
//
// Eight lanes per cell (four cells at a time per warp).  The sums are exact integer
// sums, not FP64 ones (GB300's FP64 pipe, ~1/64 of FP32, bounded the FP64
// version): each velocity component of a cell becomes the integer
// x = round(v / 2^p), 2^p = the unit in the last place of the cell's largest
// component (coarser by 2^c for cells of 1024 or more particles, so that a
// cell's sum fits in 64 bits), formed from the bits of v on the integer
// pipe.  Sums of x are exact in int64, sums of x^2 and the centred sum of
// squares in 128 bits; only the per-cell results are converted back to FP64.  The only
// rounding is each component's to the cell's resolution (at most half its
// largest ulp), the same order as one FP64 addition per term, and the result
// does not depend on the order of the sums.
#pragma once

#include "internal.cuh"

namespace dsmc {

constexpr int kSeg = 8;

// reductions over aligned segments of SEG lanes (SEG = 8 or 32)
template <int SEG = kSeg>
__device__ __forceinline__ int seg_max_i(int v) {
#pragma unroll
  for (int o = SEG / 2; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
template <int SEG = kSeg>
__device__ __forceinline__ long long seg_sum_ll(long long v) {
#pragma unroll
  for (int o = SEG / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <int SEG = kSeg>
__device__ __forceinline__ unsigned __int128 seg_sum_u128(unsigned __int128 v) {
#pragma unroll
  for (int o = SEG / 2; o > 0; o >>= 1) {
    const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
    const unsigned long long lo2 = __shfl_xor_sync(0xffffffffu, lo, o), hi2 = __shfl_xor_sync(0xffffffffu, hi, o);
    v += ((unsigned __int128)hi2 << 64) | lo2;
  }
  return v;
}

// biased exponent field of a double (2047: inf or nan)
__device__ __forceinline__ int dexp(double v) { return (__double2hiint(v) >> 20) & 0x7FF; }

// Cell scale: E = largest biased exponent of the cell's components, c the
// coarsening for large cells; the integer unit is 2^(E - 1075 + c).
struct FixScale {
  int E, c;
};

__device__ __forceinline__ FixScale cell_scale(int E, int32_t N) {
  const int bits = 32 - __clz(N > 0 ? N : 1);   // N < 2^bits
  return FixScale{E, bits > 10 ? bits - 10 : 0};
}

// round(v / unit) for the cell's unit (integer pipe only)
__device__ __forceinline__ long long to_fix(double v, const FixScale& f) {
  const uint32_t hi = (uint32_t)__double2hiint(v), lo = (uint32_t)__double2loint(v);
  const int e = (int)((hi >> 20) & 0x7FFu);
  if (e == 0) return 0;  // zero (or subnormal: below any normal cell's unit)
  const unsigned long long m = ((unsigned long long)((hi & 0xFFFFFu) | 0x100000u) << 32) | lo;
  const int sh = f.E - e + f.c;
  unsigned long long x;
  if (sh <= 0) x = m;
  else if (sh >= 64) x = 0;
  else x = (m + (1ull << (sh - 1))) >> sh;
  return (hi & 0x80000000u) ? -(long long)x : (long long)x;
}

// round(s / n) for n > 0
__device__ __forceinline__ long long div_round(long long s, long long n) {
  return s >= 0 ? (s + n / 2) / n : -((-s + n / 2) / n);
}

// The exact integer moments of one cell (8 lanes): sums and centred sum of
// squares in the cell's integer unit.  Two passes over the cell: the largest
// exponent, then the sums of x and of x^2; the centred sum follows exactly
// from sum (x - m)^2 = sum x^2 - m (2 sum x - n m) in 128-bit integers.
struct CellFix {
  FixScale f;
  long long sx, sy, sz, mx, my, mz;  // sums and rounded means (integer units)
  unsigned __int128 th;              // sum of squared deviations (units^2)
};

__device__ __forceinline__ unsigned __int128 sq128(long long x) {
  const unsigned long long u = (unsigned long long)(x < 0 ? -x : x);
  return (unsigned __int128)u * u;
}

template <int SEG = kSeg>
__device__ __forceinline__ CellFix cell_fix(const double* __restrict__ vx, const double* __restrict__ vy,
                                            const double* __restrict__ vz, int32_t a, int32_t b, int sl) {
  CellFix C;
  int E = 0;
#pragma unroll 4
  for (int32_t i = a + sl; i < b; i += SEG) E = max(E, max(dexp(vx[i]), max(dexp(vy[i]), dexp(vz[i]))));
  C.f = cell_scale(seg_max_i<SEG>(E), b - a);
  long long sx = 0, sy = 0, sz = 0;
  unsigned __int128 s2 = 0;
#pragma unroll 4
  for (int32_t i = a + sl; i < b; i += SEG) {
    const long long x = to_fix(vx[i], C.f), y = to_fix(vy[i], C.f), z = to_fix(vz[i], C.f);
    sx += x; sy += y; sz += z;
    s2 += sq128(x) + sq128(y) + sq128(z);
  }
  C.sx = seg_sum_ll<SEG>(sx); C.sy = seg_sum_ll<SEG>(sy); C.sz = seg_sum_ll<SEG>(sz);
  s2 = seg_sum_u128<SEG>(s2);
  const long long n = b - a;
  C.mx = n > 0 ? div_round(C.sx, n) : 0;
  C.my = n > 0 ? div_round(C.sy, n) : 0;
  C.mz = n > 0 ? div_round(C.sz, n) : 0;
  const __int128 corr = (__int128)C.mx * (2 * (__int128)C.sx - (__int128)n * C.mx) +
                        (__int128)C.my * (2 * (__int128)C.sy - (__int128)n * C.my) +
                        (__int128)C.mz * (2 * (__int128)C.sz - (__int128)n * C.mz);
  C.th = s2 - (unsigned __int128)corr;
  return C;
}

// ---- split integer accumulation (the block-staged cell kernels)
// The same exact moments with cheaper sums of squares: x = round(v/unit)
// is split as x = h 2^s + l (l < 2^s) and the cell accumulates the 64-bit
// sums A = sum h^2, B = sum h l and L = sum l^2 (one 32 x 32 -> 64 bit
// multiply-add each), so that sum x^2 = A 2^(2s) + B 2^(s+1) + L exactly.
// With N < 2^bits particles and |x| <= 2^(53-c) (c = max(0, bits - 10)):
// A < 2^(126-bits-2s) and L < 2^(bits+2s) both fit in 64 bits for
// s = 26 (bits <= 10) and s = (63 - bits) / 2 (bits >= 11); B < 2^63 and
// the signed sums of x stay below 2^63 as before.
__device__ __forceinline__ int fix_split(int32_t n) {
  const int bits = 32 - __clz(n > 0 ? n : 1);
  return bits <= 10 ? 26 : (63 - bits) >> 1;
}

struct FixAcc {
  long long sx, sy, sz;
  unsigned long long A, B, L;
};

// v added to the sums with integer unit 2^(Ec - 1075) (Ec = E + c)
__device__ __forceinline__ void fix_add(FixAcc& q, long long& sc, double v, int Ec, int s) {
  const uint32_t hi = (uint32_t)__double2hiint(v), lo = (uint32_t)__double2loint(v);
  const int e = (int)((hi >> 20) & 0x7FFu);
  const int sh = Ec - e;
  const unsigned long long m = ((unsigned long long)((hi & 0xFFFFFu) | 0x100000u) << 32) | lo;
  unsigned long long x;
  if (e == 0 || sh >= 64) x = 0;
  else if (sh <= 0) x = m;
  else x = ((m >> (sh - 1)) + 1) >> 1;   // = (m + 2^(sh-1)) >> sh
  sc += (hi & 0x80000000u) ? -(long long)x : (long long)x;
  const uint32_t h = (uint32_t)(x >> s), l = (uint32_t)x & ((1u << s) - 1u);
  q.A += (unsigned long long)h * h;
  q.B += (unsigned long long)h * l;
  q.L += (unsigned long long)l * l;
}

// The cell's moments from its reduced sums (the tail of cell_fix).
__device__ __forceinline__ CellFix cellfix_from(int E, int32_t n, const FixAcc& q) {
  CellFix C;
  C.f = cell_scale(E, n);
  const int s = fix_split(n);
  C.sx = q.sx; C.sy = q.sy; C.sz = q.sz;
  const unsigned __int128 s2 = ((unsigned __int128)q.A << (2 * s)) + ((unsigned __int128)q.B << (s + 1)) +
                               (unsigned __int128)q.L;
  const long long nn = n;
  C.mx = nn > 0 ? div_round(C.sx, nn) : 0;
  C.my = nn > 0 ? div_round(C.sy, nn) : 0;
  C.mz = nn > 0 ? div_round(C.sz, nn) : 0;
  const __int128 corr = (__int128)C.mx * (2 * (__int128)C.sx - (__int128)nn * C.mx) +
                        (__int128)C.my * (2 * (__int128)C.sy - (__int128)nn * C.my) +
                        (__int128)C.mz * (2 * (__int128)C.sz - (__int128)nn * C.mz);
  C.th = s2 - (unsigned __int128)corr;
  return C;
}

__device__ __forceinline__ double th_double(unsigned __int128 v) {
  return fma((double)(unsigned long long)(v >> 64), 18446744073709551616.0, (double)(unsigned long long)v);
}

// 2^(E - 1075 + c) built from its bits (integer pipe): normal for
// E + c > 52, else subnormal
__device__ __forceinline__ double unit_bits(const FixScale& f) {
  const int e = f.E + f.c - 52;  // biased exponent of the unit
  return e > 0 ? __longlong_as_double((long long)e << 52) : __longlong_as_double(1ll << (f.E + f.c - 1));
}

// Lane sl < 5 of a cell's eight writes its moment: lanes 0..2 the momentum
// sums, lane 3 Theta, lane 4 N (mk = the cell's five slots N, sum vx, sum
// vy, sum vz, Theta).
__device__ __forceinline__ void moment_store(const CellFix& C, int32_t n, int sl, double* mk, int* status) {
  if (sl == 0 && C.f.E == 0x7FF) set_status(status, DSMC_ERR_NONFINITE);
  const double unit = unit_bits(C.f);
  const long long sc = sl == 0 ? C.sx : sl == 1 ? C.sy : C.sz;
  double val;
  if (sl < 3) val = (double)sc * unit;
  else if (sl == 3) val = th_double(C.th) * unit * unit;
  else val = (double)n;
  mk[sl < 4 ? 1 + sl : 0] = val;
}

// Moment matching (Sec. 2.5, centred) of a cell of n particles: v <- alpha v
// + o with alpha = sqrt(Th_pre/Th_post) (1 if n < 2 or Th_post = 0) and o =
// u_pre - alpha u_post for component (sl < 3 ? sl : 0); C: the post-collision
// moments, mk: the pre-collision ones.
__device__ __forceinline__ void match_coeffs(const CellFix& C, int32_t n, int sl, const double* mk, double* alpha,
                                             double* o) {
  *alpha = 1.0;
  *o = 0.0;
  if (n > 0) {
    const int cmp = sl < 3 ? sl : 0;
    const double unit = unit_bits(C.f), inv = 1.0 / (double)n;
    const long long sc = cmp == 0 ? C.sx : cmp == 1 ? C.sy : C.sz;
    const double u = (double)sc * unit * inv;
    const double th = th_double(C.th) * unit * unit;
    *alpha = (n >= 2 && th > 0.0) ? sqrt(mk[4] / th) : 1.0;
    *o = mk[1 + cmp] * inv - *alpha * u;
  }
}

// The three offsets of match_coeffs at once (the same arithmetic per
// component, alpha formed once): o[c] for components c = 0, 1, 2.
__device__ __forceinline__ void match_coeffs3(const CellFix& C, int32_t n, const double* mk, double* alpha,
                                              double o[3]) {
  *alpha = 1.0;
  o[0] = o[1] = o[2] = 0.0;
  if (n > 0) {
    const double unit = unit_bits(C.f), inv = 1.0 / (double)n;
    const double th = th_double(C.th) * unit * unit;
    *alpha = (n >= 2 && th > 0.0) ? sqrt(mk[4] / th) : 1.0;
    const long long sc[3] = {C.sx, C.sy, C.sz};
#pragma unroll
    for (int cmp = 0; cmp < 3; ++cmp) {
      const double u = (double)sc[cmp] * unit * inv;
      o[cmp] = mk[1 + cmp] * inv - *alpha * u;
    }
  }
}

}  // namespace dsmc
