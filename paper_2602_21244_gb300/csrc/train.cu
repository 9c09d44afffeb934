// Training of the neural collision operator: forward, loss, hand-written
// backward with activation recomputation, Adam (Sec. 2.6: MSE against the
// harvested post-collision state; Sec. 2.3 shell projection and pair update
// and Sec. 2.5 moment matching in the graph; Adam as in Sec. 3.4.2).
//
// Per CTA (persistent, 512 threads, one 128-pair tile at a time):
//   forward   X -> z1..z3 (tcgen05, input and activations as bf16 hi + lo),
//             y, u = y/|y|, v_r' = |v_r| u, centre-of-mass update, moment
//             matching over pseudo-cells of 16 pairs (32 particles), loss
//   backward  dL/dv_new -> closed-form moment-matching and projection
//             backward -> dz4 = dL/dy; the activations recomputed: the low
//             bf16 terms of h1 and h2 regenerated by running layers 1 and 2
//             again from the saved input and high terms, then for l = 3, 2,
//             1: z_l by an MMA from exactly the forward's operands, so every
//             recomputed z_l equals the forward's bit for bit (the stored
//             variant reads back the copy the forward wrote to global
//             memory instead),
//             dz_l = dh_l * act'(z_l), dW_l += dz_l^T h_{l-1} (MN-major
//             operands, accumulated in TMEM across the CTA's tiles),
//             dh_{l-1} = dz_l W_l (W_l read MN-major from the forward tile)
//   flush     per-CTA partial gradients to global memory; a second kernel
//             sums them over CTAs in a fixed order (deterministic)
// TMEM columns: 0..127 scratch, 128..255 dW2, 256..383 dW3, 384..415 dW1
// (hi|lo input columns), 416..431 dW4^T.
#include <cuda_bf16.h>

#include "internal.cuh"
#include "tc.cuh"

namespace dsmc {

namespace {
constexpr int kT = 128;          // pairs per tile
constexpr int kNT = 512;         // threads
constexpr int kH = 128;          // width
constexpr int kXin = 32;         // input columns (hi | lo)
constexpr int kGroup = 16;       // pairs per pseudo-cell
// shared memory layout
constexpr uint32_t S_WOUT = 0;                         // [16 x 128]
constexpr uint32_t S_WIN = S_WOUT + 16 * kH * 2;       // [128 x 32]
constexpr uint32_t S_W2 = S_WIN + kH * kXin * 2;       // [128 x 128]
constexpr uint32_t S_W3 = S_W2 + kH * kH * 2;          // [128 x 128]
constexpr uint32_t S_X = S_W3 + kH * kH * 2;           // [128 x 32] hi | lo
constexpr uint32_t S_H1 = S_X + kT * kXin * 2;         // [128 x 128] h1 (single bf16 copy)
constexpr uint32_t S_H2 = S_H1 + kT * kH * 2;          // [128 x 128] h2 (single)
constexpr uint32_t S_WK = S_H2 + kT * kH * 2;          // [128 x 128] x 2: working hi, lo; later dz
constexpr uint32_t S_WKLO = S_WK + kT * kH * 2;
constexpr uint32_t S_DZ4 = S_WKLO + kT * kH * 2;       // [128 x 16] dz of the output layer (bf16)
constexpr uint32_t S_DZ4F = S_DZ4 + kT * 16 * 2;       // [128 x 3] FP32
constexpr uint32_t S_BIAS = S_DZ4F + kT * 4 * 4;       // 3*128 + 16 floats
constexpr uint32_t S_DB = S_BIAS + (3 * kH + 16) * 4;  // 3*128 + 16 floats (bias gradients)
constexpr uint32_t S_MISC = S_DB + (3 * kH + 16) * 4;  // mbarrier, tmem ptr, flag, loss
constexpr uint32_t S_TOTAL = S_MISC + 64;
// per-CTA partial: dW1 [128 x 32], dW2, dW3 [128 x 128], dW4^T [128 x 16], then the bias
// gradients of each of the 4 TMEM lane groups [4 x 400], then the loss of each lane group
constexpr int kPDB = kH * kXin + 2 * kH * kH + kH * 16;
constexpr int kPLOSS = kPDB + 4 * 400;
constexpr int kPartial = kPLOSS + 16;
constexpr int kNW = kH * 8 + 2 * kH * kH + 3 * kH;   // weights (d_in 8)
constexpr int kNB = 3 * kH + 3;                      // biases
constexpr uint32_t TM_DW2 = 128, TM_DW3 = 256, TM_DW1 = 384, TM_DW4 = 416;
}  // namespace

struct TrainArgs {
  int mode;                  // 0 forward only, 1 backward from given dL/dv_new, 2 MSE loss vs targets
  int act;
  int64_t n;                 // pairs (multiple of 16)
  uint64_t seed, t;
  double sigma_v_inv, T_ref_inv, eps;
  const float* theta;        // FP32 parameters: weights (row-major per layer), then biases
  const double *vi, *vj, *T, *ti, *tj;   // [n x 3], [n], targets [n x 3]
  const double *gi, *gj;     // mode 1: dL/dv_new [n x 3]
  double *oi, *oj;           // mode 0: v_new [n x 3]
  float* zst;                // stored variant: z_l (accumulator, without bias) per tile, else null
  float* partial;            // [gridDim x kPartial]
  int* status;
};

__device__ __forceinline__ float act_fn(int act, float z) {
  if (act == 1) return fmaxf(z, 0.f);
  return __fdividef(z, 1.f + __expf(-z));
}
__device__ __forceinline__ float act_grad(int act, float z) {
  if (act == 1) return z > 0.f ? 1.f : 0.f;
  const float s = __fdividef(1.f, 1.f + __expf(-z));
  return s * (1.f + z * (1.f - s));
}

// sum over the 16 lanes of this half-warp (groups are 16 consecutive rows)
__device__ __forceinline__ double half_sum(double v) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// v[32] per lane -> lane l returns the sum over the warp's lanes of v[l]
__device__ __forceinline__ float warp_colsum32(float* v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int w = 16; w >= 1; w >>= 1) {
#pragma unroll
    for (int k = 0; k < w; ++k) {
      const bool hi = lane & w;
      const float send = hi ? v[k] : v[k + w];
      const float keep = hi ? v[k + w] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, w);
    }
  }
  return v[0];
}

__device__ __forceinline__ uint16_t to_bf16(float x) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

__device__ __forceinline__ void box_muller2(double u1, double u2, float* z0, float* z1) {
  const float rho = sqrtf(-2.f * __logf((float)(1.0 - u1)));
  float s, c;
  __sincosf((float)(2.0 * DSMC_PI * u2), &s, &c);
  *z0 = rho * c;
  *z1 = rho * s;
}

__device__ __forceinline__ uint64_t kdesc(uint32_t a, int K) { return tc::sdesc(a, 128, (uint32_t)(K / 8) * 128); }
// MN-major view of a [rows x F] tile: MN = F (features), K = rows
__device__ __forceinline__ uint64_t mdesc(uint32_t a, int F) { return tc::sdesc(a, (uint32_t)(F / 8) * 128, 128); }

__global__ void __launch_bounds__(kNT, 1) k_train(TrainArgs a) {
  extern __shared__ __align__(1024) char sm[];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int row = ((warp & 3) << 5) | lane, cg = warp >> 2, c0 = cg * 32;
  const uint32_t sb = tc::smem_u32(sm);
  uint64_t* mbar = (uint64_t*)(sm + S_MISC);
  uint32_t* tptr = (uint32_t*)(sm + S_MISC + 8);
  volatile int* flag = (volatile int*)(sm + S_MISC + 12);
  float* bias = (float*)(sm + S_BIAS);
  // bias gradients and loss accumulate in registers of fixed threads (no atomics,
  // so the result does not depend on warp scheduling)
  float dbacc[3] = {0.f, 0.f, 0.f};  // layer l, column c0 + lane
  float dbo[3] = {0.f, 0.f, 0.f};    // output bias (lane 0 of warps 0..3)
  double lossw = 0.0;                // loss of this warp's rows (lane 0 of warps 0..3)
  float* dz4f = (float*)(sm + S_DZ4F);
  // ---- weights into K-major tiles, biases
  {
    uint32_t* z = (uint32_t*)(sm + S_WOUT);
    for (int q = t; q < (16 * kH * 2 + kH * kXin * 2) / 4; q += kNT) z[q] = 0u;
    const float* bsrc = a.theta + kNW;
    for (int q = t; q < 3 * kH + 16; q += kNT) bias[q] = q < 3 * kH + 3 ? bsrc[q] : 0.f;
    __syncthreads();
    for (int e = t; e < kH * 8; e += kNT) {
      const int n = e >> 3, k = e & 7;
      const uint16_t wb = to_bf16(a.theta[e]);
      *(uint16_t*)(sm + S_WIN + tc::kmajor_offset(n, k, kXin)) = wb;
      *(uint16_t*)(sm + S_WIN + tc::kmajor_offset(n, 16 + k, kXin)) = wb;
    }
    const float* w2 = a.theta + kH * 8;
    for (int e = t; e < kH * kH; e += kNT) {
      *(uint16_t*)(sm + S_W2 + tc::kmajor_offset(e >> 7, e & 127, kH)) = to_bf16(w2[e]);
      *(uint16_t*)(sm + S_W3 + tc::kmajor_offset(e >> 7, e & 127, kH)) = to_bf16(w2[kH * kH + e]);
    }
    const float* w4 = w2 + 2 * kH * kH;
    for (int e = t; e < 3 * kH; e += kNT)
      *(uint16_t*)(sm + S_WOUT + tc::kmajor_offset(e >> 7, e & 127, kH)) = to_bf16(w4[e]);
  }
  if (warp == 0) { tc::tmem_alloc(tptr, 512); tc::tmem_relinquish(); }
  if (t == 0) { tc::mbar_init(mbar, 1); tc::mbar_fence_init(); }
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tm = *(volatile uint32_t*)tptr;
  const uint32_t lane_tm = tm + ((uint32_t)((warp & 3) * 32) << 16);
  uint32_t phase = 0;
  bool alive = true;
  int tiles_done = 0;

  // one elected thread commits the issued MMAs and waits; everyone syncs
  auto sync_mma = [&]() -> bool {
    if (t == 0) {
      tc::commit(mbar);
      *flag = tc::mbar_wait(mbar, phase, a.status, kBarrierLimitNs) ? 1 : 0;
    }
    __syncthreads();
    phase ^= 1u;
    tc::fence_after();
    return *flag != 0;
  };
  auto to_mma = [&]() {  // make shared-memory writes and TMEM reads visible before an MMA
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
  };

  // The MMA of hidden layer l + 1 (l = 1, 2) on its input as hi + lo terms:
  // h1 = S_H1 + S_WKLO, h2 = S_H2 + S_WK (thread 0)
  auto hidden_mma = [&](int l) {
    const uint32_t id = tc::idesc_bf16(kT, kH);
    const uint32_t wl = l == 1 ? S_W2 : S_W3, hhi = l == 1 ? S_H1 : S_H2, hlo = l == 1 ? S_WKLO : S_WK;
    for (int s = 0; s < 8; ++s)
      tc::mma_bf16(tm, kdesc(sb + hhi + 256u * s, kH), kdesc(sb + wl + 256u * s, kH), id, s > 0);
    for (int s = 0; s < 8; ++s)
      tc::mma_bf16(tm, kdesc(sb + hlo + 256u * s, kH), kdesc(sb + wl + 256u * s, kH), id, 1);
  };
  // Epilogue of hidden layer l from this thread's 32 accumulator values v:
  // bias, activation (SiLU four values at a time on the paired FP32 pipe, as
  // in the collide kernel's epilogue), the hi + lo split; hi and lo stored as
  // the next layer's input (l = 0: S_H1, S_WKLO; l = 1: S_H2, S_WK; l = 2,
  // the output layer's: S_WK, S_WKLO).  with_hi false: only the lo term
  // (the backward's regeneration; the hi terms are still in S_H1, S_H2).
  auto hidden_epilogue = [&](int l, const float* v, bool with_hi) {
    uint32_t pk[16], lo[16];
    const float2* b2 = (const float2*)(bias + l * kH + c0);
#pragma unroll
    for (int q = 0; q < 16; q += 2) {
      float2 va = __fadd2_rn(make_float2(v[2 * q], v[2 * q + 1]), b2[q]);
      float2 vb = __fadd2_rn(make_float2(v[2 * q + 2], v[2 * q + 3]), b2[q + 1]);
      if (a.act == 0) {
        tc::silu4x2(va, vb);
      } else {
        va = make_float2(act_fn(a.act, va.x), act_fn(a.act, va.y));
        vb = make_float2(act_fn(a.act, vb.x), act_fn(a.act, vb.y));
      }
      const float2 m1 = make_float2(-1.f, -1.f);
      pk[q] = tc::pack_bf16x2(va.x, va.y);
      pk[q + 1] = tc::pack_bf16x2(vb.x, vb.y);
      const float2 ra = __ffma2_rn(make_float2(__uint_as_float(pk[q] << 16), __uint_as_float(pk[q] & 0xFFFF0000u)), m1, va);
      const float2 rb = __ffma2_rn(make_float2(__uint_as_float(pk[q + 1] << 16), __uint_as_float(pk[q + 1] & 0xFFFF0000u)),
                                   m1, vb);
      lo[q] = tc::pack_bf16x2(ra.x, ra.y);
      lo[q + 1] = tc::pack_bf16x2(rb.x, rb.y);
    }
    const uint32_t dhi = l == 0 ? S_H1 : l == 1 ? S_H2 : S_WK, dlo = l == 1 ? S_WK : S_WKLO;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t off = tc::kmajor_offset(row, c0 + 8 * j, kH);
      if (with_hi) tc::st_shared_v4(sb + dhi + off, pk[4 * j], pk[4 * j + 1], pk[4 * j + 2], pk[4 * j + 3]);
      tc::st_shared_v4(sb + dlo + off, lo[4 * j], lo[4 * j + 1], lo[4 * j + 2], lo[4 * j + 3]);
    }
  };

  const int64_t ntiles = (a.n + kT - 1) / kT;
  for (int64_t tile = blockIdx.x; tile < ntiles && alive; tile += gridDim.x) {
    const int64_t p = tile * kT + row;
    const bool rowthr = t < kT;
    const bool valid = rowthr && p < a.n;
    double vi[3] = {0, 0, 0}, vj[3] = {0, 0, 0};
    // ---------------- features (rows)
    if (rowthr) {
      float f[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) f[q] = 0.f;
      if (valid) {
        for (int c = 0; c < 3; ++c) { vi[c] = a.vi[3 * p + c]; vj[c] = a.vj[3 * p + c]; }
        f[0] = (float)((vi[0] - vj[0]) * a.sigma_v_inv);
        f[1] = (float)((vi[1] - vj[1]) * a.sigma_v_inv);
        f[2] = (float)((vi[2] - vj[2]) * a.sigma_v_inv);
        f[3] = (float)(a.T[p] * a.T_ref_inv);
        const u32x4 wa = draw(a.seed, (uint32_t)p, 0u, a.t, TAG_NOISE, 0);
        const u32x4 wb = draw(a.seed, (uint32_t)p, 0u, a.t, TAG_NOISE, 1);
        box_muller2(u53(wa.x, wa.y), u53(wa.z, wa.w), &f[4], &f[5]);
        box_muller2(u53(wb.x, wb.y), u53(wb.z, wb.w), &f[6], &f[7]);
      }
      uint32_t hi[8], lo[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        hi[q] = tc::pack_bf16x2(f[2 * q], f[2 * q + 1]);
        lo[q] = tc::pack_bf16x2(f[2 * q] - __uint_as_float(hi[q] << 16), f[2 * q + 1] - __uint_as_float(hi[q] & 0xFFFF0000u));
      }
      tc::st_shared_v4(sb + S_X + tc::kmajor_offset(row, 0, kXin), hi[0], hi[1], hi[2], hi[3]);
      tc::st_shared_v4(sb + S_X + tc::kmajor_offset(row, 8, kXin), hi[4], hi[5], hi[6], hi[7]);
      tc::st_shared_v4(sb + S_X + tc::kmajor_offset(row, 16, kXin), lo[0], lo[1], lo[2], lo[3]);
      tc::st_shared_v4(sb + S_X + tc::kmajor_offset(row, 24, kXin), lo[4], lo[5], lo[6], lo[7]);
    }
    to_mma();
    // ---------------- forward, layers 1..3 (scratch accumulator at TMEM column 0)
    for (int l = 0; l < 3 && alive; ++l) {
      if (t == 0) {
        tc::fence_after();
        const uint32_t id = tc::idesc_bf16(kT, kH);
        if (l == 0) {
          for (int s = 0; s < 2; ++s)
            tc::mma_bf16(tm, kdesc(sb + S_X + 256u * s, kXin), kdesc(sb + S_WIN + 256u * s, kXin), id, s > 0);
        } else {
          hidden_mma(l);
        }
      }
      if (!sync_mma()) { alive = false; break; }
      float v[32];
      tc::ld32(lane_tm + (uint32_t)c0, v);
      if (a.zst && a.mode != 0) {   // stored variant: this tile's z_l, row-major [128 x 128]
        float4* dst = (float4*)(a.zst + (((size_t)tile * 3 + l) * kT + row) * kH + c0);
#pragma unroll
        for (int q = 0; q < 8; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      }
      hidden_epilogue(l, v, true);
      to_mma();
    }
    if (!alive) break;
    // ---------------- output layer
    if (t == 0) {
      tc::fence_after();
      const uint32_t id = tc::idesc_bf16(kT, 16);
      for (int s = 0; s < 8; ++s)
        tc::mma_bf16(tm, kdesc(sb + S_WK + 256u * s, kH), kdesc(sb + S_WOUT + 256u * s, kH), id, s > 0);
      for (int s = 0; s < 8; ++s)
        tc::mma_bf16(tm, kdesc(sb + S_WKLO + 256u * s, kH), kdesc(sb + S_WOUT + 256u * s, kH), id, 1);
    }
    if (!sync_mma()) { alive = false; break; }
    float y[3] = {0.f, 0.f, 0.f};
    if (cg == 0) {
      float v[16];
      tc::ld16(lane_tm, v);
      y[0] = v[0] + bias[3 * kH]; y[1] = v[1] + bias[3 * kH + 1]; y[2] = v[2] + bias[3 * kH + 2];
    }
    // ---------------- shell projection, pair update, moment matching, loss (rows)
    if (rowthr) {
      double ur[3], g = 0.0, ny = 0.0, u[3], pi[3], pj[3];
      for (int c = 0; c < 3; ++c) ur[c] = vi[c] - vj[c];
      g = sqrt(ur[0] * ur[0] + ur[1] * ur[1] + ur[2] * ur[2]);
      const double yd[3] = {y[0], y[1], y[2]};
      ny = sqrt(yd[0] * yd[0] + yd[1] * yd[1] + yd[2] * yd[2]);
      const double iny = valid && ny > 0.0 ? 1.0 / ny : 0.0;
      for (int c = 0; c < 3; ++c) {
        u[c] = yd[c] * iny;
        const double cm = 0.5 * (vi[c] + vj[c]);
        pi[c] = cm + 0.5 * g * u[c];
        pj[c] = cm - 0.5 * g * u[c];
      }
      // group moments over the 32 particles of the pseudo-cell (two passes)
      double upre[3], upost[3], thpre = 0.0, thpost = 0.0;
      for (int c = 0; c < 3; ++c) {
        upre[c] = half_sum(vi[c] + vj[c]) * (1.0 / (2 * kGroup));
        upost[c] = half_sum(pi[c] + pj[c]) * (1.0 / (2 * kGroup));
      }
      double dpi[3], dpj[3], tpre = 0.0, tpost = 0.0;
      for (int c = 0; c < 3; ++c) {
        const double a1 = vi[c] - upre[c], a2 = vj[c] - upre[c];
        tpre += a1 * a1 + a2 * a2;
        dpi[c] = pi[c] - upost[c];
        dpj[c] = pj[c] - upost[c];
        tpost += dpi[c] * dpi[c] + dpj[c] * dpj[c];
      }
      thpre = half_sum(tpre);
      thpost = half_sum(tpost);
      const double alpha = thpost > 0.0 ? sqrt(thpre / thpost) : 1.0;
      double ni[3], nj[3];
      for (int c = 0; c < 3; ++c) { ni[c] = upre[c] + alpha * dpi[c]; nj[c] = upre[c] + alpha * dpj[c]; }
      if (a.mode == 0) {
        if (valid) for (int c = 0; c < 3; ++c) { a.oi[3 * p + c] = ni[c]; a.oj[3 * p + c] = nj[c]; }
      } else {
        double Gi[3] = {0, 0, 0}, Gj[3] = {0, 0, 0};
        double l2 = 0.0;
        if (valid) {
          if (a.mode == 2) {
            const double sc = a.sigma_v_inv * a.sigma_v_inv / (double)a.n;
            for (int c = 0; c < 3; ++c) {
              const double ri = ni[c] - a.ti[3 * p + c], rj = nj[c] - a.tj[3 * p + c];
              l2 += ri * ri + rj * rj;
              Gi[c] = ri * sc;
              Gj[c] = rj * sc;
            }
          } else {
            for (int c = 0; c < 3; ++c) { Gi[c] = a.gi[3 * p + c]; Gj[c] = a.gj[3 * p + c]; }
          }
        }
        if (a.mode == 2) {  // loss = sum |v_new - v_target|^2 / sigma_v^2 / (2 n)
          double lw = l2 * a.sigma_v_inv * a.sigma_v_inv / (2.0 * (double)a.n);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) lw += __shfl_xor_sync(0xffffffffu, lw, o);
          lossw += lw;
        }
        // moment-matching backward: dL/dv = alpha (G - Gbar) - (alpha S / Theta_post) (v - u_post)
        double gbar[3], S = 0.0;
        for (int c = 0; c < 3; ++c) gbar[c] = half_sum(Gi[c] + Gj[c]) * (1.0 / (2 * kGroup));
        double sl = 0.0;
        for (int c = 0; c < 3; ++c) sl += Gi[c] * dpi[c] + Gj[c] * dpj[c];
        S = half_sum(sl);
        const double k2 = thpost > 0.0 ? alpha * S / thpost : 0.0;
        double dvr[3], ud = 0.0;
        for (int c = 0; c < 3; ++c) {
          const double di = alpha * (Gi[c] - gbar[c]) - k2 * dpi[c];
          const double dj = alpha * (Gj[c] - gbar[c]) - k2 * dpj[c];
          dvr[c] = 0.5 * (di - dj);   // v_r' enters as +1/2 for i, -1/2 for j
          ud += u[c] * dvr[c];
        }
        // projection backward: dy = (g/|y|)(I - u u^T) dv_r'
        const double s = valid ? g * iny : 0.0;
        for (int c = 0; c < 3; ++c) dz4f[4 * row + c] = valid ? (float)(s * (dvr[c] - u[c] * ud)) : 0.f;
        uint32_t d0 = tc::pack_bf16x2(dz4f[4 * row], dz4f[4 * row + 1]);
        uint32_t d1 = tc::pack_bf16x2(dz4f[4 * row + 2], 0.f);
        tc::st_shared_v4(sb + S_DZ4 + tc::kmajor_offset(row, 0, 16), d0, d1, 0u, 0u);
        tc::st_shared_v4(sb + S_DZ4 + tc::kmajor_offset(row, 8, 16), 0u, 0u, 0u, 0u);
      }
    }
    if (a.mode == 0) { tc::fence_before(); __syncthreads(); tc::fence_after(); continue; }
    // bias gradient of the output layer
    if (t < kT) {
      float v3[3] = {dz4f[4 * row], dz4f[4 * row + 1], dz4f[4 * row + 2]};
      for (int c = 0; c < 3; ++c) {
        float s3 = v3[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s3 += __shfl_xor_sync(0xffffffffu, s3, o);
        dbo[c] += s3;
      }
    }
    to_mma();
    // ---------------- dW4^T += h3^T dz4 (hi and lo), and z3 recomputed from h2
    const uint32_t acc0 = tiles_done > 0 ? 1u : 0u;
    if (t == 0) {
      tc::fence_after();
      const uint32_t id4 = tc::idesc_bf16(kT, 16) | (1u << 15) | (1u << 16);
      for (int s = 0; s < 8; ++s)
        tc::mma_bf16(tm + TM_DW4, mdesc(sb + S_WK + 2u * 2048u * s, kH), mdesc(sb + S_DZ4 + 2u * 256u * s, 16), id4,
                     (acc0 | (s > 0)) ? 1u : 0u);
      for (int s = 0; s < 8; ++s)
        tc::mma_bf16(tm + TM_DW4, mdesc(sb + S_WKLO + 2u * 2048u * s, kH), mdesc(sb + S_DZ4 + 2u * 256u * s, 16), id4, 1);
      if (!a.zst) {   // regeneration starts with z1 from x (hi + lo)
        const uint32_t id = tc::idesc_bf16(kT, kH);
        for (int s = 0; s < 2; ++s)
          tc::mma_bf16(tm, kdesc(sb + S_X + 256u * s, kXin), kdesc(sb + S_WIN + 256u * s, kXin), id, s > 0);
      }
    }
    if (!sync_mma()) { alive = false; break; }
    if (!a.zst) {
      // h1 and h2 low terms regenerated (the forward's arithmetic on the same
      // accumulators), then z3 = W3 (h2 hi + lo): all equal to the forward's
      for (int l = 0; l < 2 && alive; ++l) {
        float v[32];
        tc::ld32(lane_tm + (uint32_t)c0, v);
        hidden_epilogue(l, v, false);
        to_mma();
        if (t == 0) {
          tc::fence_after();
          hidden_mma(l + 1);
        }
        if (!sync_mma()) alive = false;
      }
      if (!alive) break;
    }
    // dh3 = dz4 W4 on CUDA cores (K = 3), dz3 = dh3 * act'(z3)
    float dh[32];
    {
#pragma unroll
      for (int q = 0; q < 32; ++q) dh[q] = 0.f;
      const float d0 = dz4f[4 * row], d1 = dz4f[4 * row + 1], d2 = dz4f[4 * row + 2];
      for (int q = 0; q < 32; ++q) {
        const int k = c0 + q;
        const float w0 = __uint_as_float((uint32_t)(*(const uint16_t*)(sm + S_WOUT + tc::kmajor_offset(0, k, kH))) << 16);
        const float w1 = __uint_as_float((uint32_t)(*(const uint16_t*)(sm + S_WOUT + tc::kmajor_offset(1, k, kH))) << 16);
        const float w2 = __uint_as_float((uint32_t)(*(const uint16_t*)(sm + S_WOUT + tc::kmajor_offset(2, k, kH))) << 16);
        dh[q] = d0 * w0 + d1 * w1 + d2 * w2;
      }
    }
    // layers 3, 2, 1
    for (int l = 2; l >= 0 && alive; --l) {
      float z[32];
      if (a.zst) {
        const float4* src = (const float4*)(a.zst + (((size_t)tile * 3 + l) * kT + row) * kH + c0);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float4 f = src[q];
          z[4 * q] = f.x; z[4 * q + 1] = f.y; z[4 * q + 2] = f.z; z[4 * q + 3] = f.w;
        }
      } else {
        tc::ld32(lane_tm + (uint32_t)c0, z);
      }
      float dz[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) dz[q] = dh[q] * act_grad(a.act, z[q] + bias[l * kH + c0 + q]);
      uint32_t pk[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) pk[q] = tc::pack_bf16x2(dz[2 * q], dz[2 * q + 1]);
#pragma unroll
      for (int j = 0; j < 4; ++j)
        tc::st_shared_v4(sb + S_WK + tc::kmajor_offset(row, c0 + 8 * j, kH), pk[4 * j], pk[4 * j + 1], pk[4 * j + 2],
                         pk[4 * j + 3]);
      dbacc[l] += warp_colsum32(dz);
      to_mma();
      // dW_l += dz^T h_{l-1}; dh_{l-1} = dz W_l (not needed for l = 0)
      if (t == 0) {
        tc::fence_after();
        if (l > 0) {
          const uint32_t hprev = l == 2 ? S_H2 : S_H1;
          const uint32_t wl = l == 2 ? S_W3 : S_W2;
          const uint32_t dw = l == 2 ? TM_DW3 : TM_DW2;
          const uint32_t idw = tc::idesc_bf16(kH, kH) | (1u << 15) | (1u << 16);
          for (int s = 0; s < 8; ++s)
            tc::mma_bf16(tm + dw, mdesc(sb + S_WK + 2u * 2048u * s, kH), mdesc(sb + hprev + 2u * 2048u * s, kH), idw,
                         (acc0 | (s > 0)) ? 1u : 0u);
          const uint32_t idh = tc::idesc_bf16(kT, kH) | (1u << 16);
          for (int s = 0; s < 8; ++s)
            tc::mma_bf16(tm, kdesc(sb + S_WK + 256u * s, kH), mdesc(sb + wl + 2u * 2048u * s, kH), idh, s > 0);
        } else {
          const uint32_t idw = tc::idesc_bf16(kH, kXin) | (1u << 15) | (1u << 16);
          for (int s = 0; s < 8; ++s)
            tc::mma_bf16(tm + TM_DW1, mdesc(sb + S_WK + 2u * 2048u * s, kH), mdesc(sb + S_X + 2u * 512u * s, kXin), idw,
                         (acc0 | (s > 0)) ? 1u : 0u);
        }
      }
      if (!sync_mma()) { alive = false; break; }
      if (l == 0) break;
      tc::ld32(lane_tm + (uint32_t)c0, dh);
      tc::fence_before();
      __syncthreads();
      if (a.zst) continue;   // the stored variant reads z_{l-1} back
      // z_{l-1} recomputed from the forward's own operands: h1 (hi + lo, the
      // low terms regenerated above and still in S_WKLO) for layer 2, x (hi
      // + lo) for layer 1
      if (t == 0) {
        tc::fence_after();
        const uint32_t id = tc::idesc_bf16(kT, kH);
        if (l == 2) {
          hidden_mma(1);
        } else {
          for (int s = 0; s < 2; ++s)
            tc::mma_bf16(tm, kdesc(sb + S_X + 256u * s, kXin), kdesc(sb + S_WIN + 256u * s, kXin), id, s > 0);
        }
      }
      if (!sync_mma()) { alive = false; break; }
    }
    ++tiles_done;
    tc::fence_before();
    __syncthreads();
  }
  // ---------------- flush this CTA's partial gradients
  if (alive && a.mode != 0) {
    float* P = a.partial + (size_t)blockIdx.x * kPartial;
    if (tiles_done == 0) {
      for (int q = t; q < kPartial; q += kNT) P[q] = 0.f;
    } else {
      float v[32];
      // dW2, dW3: [128 out x 128 in]
      tc::ld32(lane_tm + TM_DW2 + (uint32_t)c0, v);
      for (int q = 0; q < 32; ++q) P[kH * kXin + row * kH + c0 + q] = v[q];
      tc::ld32(lane_tm + TM_DW3 + (uint32_t)c0, v);
      for (int q = 0; q < 32; ++q) P[kH * kXin + kH * kH + row * kH + c0 + q] = v[q];
      if (cg == 0) {
        tc::ld32(lane_tm + TM_DW1, v);  // [128 out x 32 (hi | lo)]
        for (int q = 0; q < 32; ++q) P[row * kXin + q] = v[q];
        float w4[16];
        tc::ld16(lane_tm + TM_DW4, w4);  // [128 in x 16 out]
        for (int q = 0; q < 16; ++q) P[kH * kXin + 2 * kH * kH + row * 16 + q] = w4[q];
      }
      const int g = warp & 3;
      for (int l = 0; l < 3; ++l) P[kPDB + g * 400 + l * kH + c0 + lane] = dbacc[l];
      if (cg == 0 && lane == 0) {
        for (int c = 0; c < 3; ++c) P[kPDB + g * 400 + 3 * kH + c] = dbo[c];
        P[kPLOSS + g] = (float)lossw;
      }
    }
  } else if (a.mode != 0 && t == 0 && !alive) {
    set_status(a.status, DSMC_ERR_TIMEOUT);
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 0) tc::tmem_dealloc(tm, 512);
}

// Sum the per-CTA partials in CTA order; write gradients in the weight layout
// (row-major per layer, then biases) and the loss.
__global__ void k_train_reduce(const float* __restrict__ partial, int nblk, int d_in, float* __restrict__ grad,
                               double* loss) {
  const int nw = kH * d_in + 2 * kH * kH + 3 * kH;
  const int nb = kNB;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nw + nb + 1; q += gridDim.x * blockDim.x) {
    float s = 0.f;
    if (q < kH * d_in) {                       // W1[o][k] = hi column k + lo column 16 + k
      const int o = q / d_in, k = q % d_in;
      for (int b = 0; b < nblk; ++b) s += partial[(size_t)b * kPartial + o * kXin + k] + partial[(size_t)b * kPartial + o * kXin + 16 + k];
    } else if (q < kH * d_in + 2 * kH * kH) {  // W2, W3
      const int r = q - kH * d_in;
      for (int b = 0; b < nblk; ++b) s += partial[(size_t)b * kPartial + kH * kXin + r];
    } else if (q < nw) {                       // W4[o][k] = dW4^T[k][o]
      const int r = q - kH * d_in - 2 * kH * kH, o = r / kH, k = r % kH;
      for (int b = 0; b < nblk; ++b) s += partial[(size_t)b * kPartial + kH * kXin + 2 * kH * kH + k * 16 + o];
    } else if (q < nw + nb) {                  // biases: lane groups 0..3 of every CTA, in order
      const int r = q - nw;
      for (int b = 0; b < nblk; ++b)
        for (int g = 0; g < 4; ++g) s += partial[(size_t)b * kPartial + kPDB + g * 400 + r];
    } else {
      double l = 0.0;
      for (int b = 0; b < nblk; ++b)
        for (int g = 0; g < 4; ++g) l += partial[(size_t)b * kPartial + kPLOSS + g];
      if (loss) *loss = l;
      continue;
    }
    grad[q] = s;
  }
}

// Adam (Kingma & Ba 2015, Algorithm 1) on FP32 parameters theta = [weights, biases];
// optionally writes the bf16 weights and FP32 biases the collide kernel takes.
__global__ void k_adam(int n_w, int n_b, const float* __restrict__ grad, float* __restrict__ master,
                       float* __restrict__ m, float* __restrict__ v, uint16_t* __restrict__ w_bf16,
                       float* __restrict__ bias, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n_w + n_b; q += gridDim.x * blockDim.x) {
    const float g = grad[q];
    const float mq = b1 * m[q] + (1.f - b1) * g;
    const float vq = b2 * v[q] + (1.f - b2) * g * g;
    m[q] = mq;
    v[q] = vq;
    const float th = master[q] - lr * (mq * c1) / (sqrtf(vq * c2) + eps);
    master[q] = th;
    if (q < n_w) {
      if (w_bf16) w_bf16[q] = to_bf16(th);
    } else if (bias) {
      bias[q - n_w] = th;
    }
  }
}

size_t train_act_bytes(int64_t n) { return sizeof(float) * 3 * (size_t)kT * kH * (size_t)((n + kT - 1) / kT); }

size_t train_ws(int sms) { return align256(sizeof(float) * (size_t)kPartial * (size_t)(sms > 0 ? sms : 1)); }

int launch_train(Ctx* c, const dsmc_mlp_t& mlp, int mode, uint64_t seed, uint64_t t, int64_t n,
                 const float* theta, const double* vi, const double* vj, const double* T,
                 const double* ti, const double* tj, const double* gi, const double* gj, double* oi, double* oj,
                 float* grad, double* loss, void* ws, size_t ws_bytes, cudaStream_t s, float* act) {
  const int sms = sm_count(c);
  if (mode != 0 && ws_bytes < train_ws(sms)) return record(c, DSMC_ERR_ARG, "train: workspace too small");
  if (cudaFuncSetAttribute((const void*)k_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S_TOTAL) !=
      cudaSuccess)
    return record(c, DSMC_ERR_CUDA, "train: shared-memory attribute");
  TrainArgs a;
  a.mode = mode; a.act = mlp.act; a.n = n; a.seed = seed; a.t = t;
  a.sigma_v_inv = 1.0 / mlp.sigma_v; a.T_ref_inv = 1.0 / mlp.T_ref; a.eps = mlp.eps;
  a.theta = theta; a.vi = vi; a.vj = vj; a.T = T; a.ti = ti; a.tj = tj; a.gi = gi; a.gj = gj;
  a.oi = oi; a.oj = oj; a.zst = act; a.partial = (float*)ws; a.status = status_ptr(c);
  const int64_t tiles = (n + kT - 1) / kT;
  const int blocks = (int)(tiles < sms ? (tiles > 0 ? tiles : 1) : sms);
  k_train<<<blocks, kNT, S_TOTAL, s>>>(a);
  count_launches(c, 1);
  if (mode != 0) {
    k_train_reduce<<<64, 256, 0, s>>>((const float*)ws, blocks, mlp.d_in, grad, loss);
    count_launches(c, 1);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : DSMC_ERR_CUDA;
}

int launch_adam(Ctx* c, int n_w, int n_b, const float* grad, float* master, float* m, float* v, uint16_t* w,
                float* bias, float lr, double b1, double b2, double eps, int64_t step, cudaStream_t s) {
  const float c1 = (float)(1.0 / (1.0 - pow(b1, (double)step)));
  const float c2 = (float)(1.0 / (1.0 - pow(b2, (double)step)));
  k_adam<<<64, 256, 0, s>>>(n_w, n_b, grad, master, m, v, w, bias, lr, (float)b1, (float)b2, (float)eps, c1, c2);
  count_launches(c, 1);
  return cudaGetLastError() == cudaSuccess ? 0 : DSMC_ERR_CUDA;
}

}  // namespace dsmc
