// Neural collision operator (Sec. 2.2-2.3) on the tcgen05 tensor cores.
//
// A CTA of 512 threads runs two warp groups of 8 warps, each owning a tile
// of 128 pairs and 256 TMEM columns (the FP32 accumulator, then the next
// layer's A operand), so that one group's feature build, activation epilogue
// and pair update run while the tensor core works on the other group's layer
// (ping-pong; a single 16-warp group when two slots do not fit).  Within a
// group: thread t < 128 builds row t of the bf16 input tile X (shared
// memory), one elected thread issues the layer's tcgen05.mma chain (FP32
// accumulator in TMEM, the bias added by the MMAs) and waits on the group's
// mbarrier, the group's warps read their 32 TMEM lanes back (tcgen05.ld),
// apply the activation and write the next layer's A operand into tensor memory
// (tcgen05.st; row m in lane m, two bf16 per column) as two bf16 terms
// (hi = bf16(a), lo = bf16(a - hi)) multiplied by the same bf16 weights:
// bf16 operands, FP32 accumulation, about 16 significant bits kept for the
// activations (single bf16 storage costs up to 6e-2 in the output direction
// of badly conditioned pairs).  A hidden layer's MMA thus reads only its
// weights from shared memory (with A there too its operand reads ran near
// the SM's shared-memory bandwidth).  The weights of all layers stay in
// shared memory for the life of the CTA.  After the last layer thread t
// projects y onto the energy shell and applies the centre-of-mass update of
// its pair in FP64.
//
// The collide kernel is persistent: each group claims 128-pair tiles of one
// round at a time from a global cursor, in round-major order, and a row
// waits (bounded) until the previous pairs of its two particles are done
// (per-particle done stamps), so no grid-wide barrier separates the rounds.
#include <cstdio>

#include "internal.cuh"
#include "tc.cuh"

namespace dsmc {

constexpr int kTileM = 128;
constexpr int kThreads = 512;    // 16 warps: 4 per TMEM lane group, splitting the columns
constexpr int kWidth = 128;
constexpr int kKin = 32;         // input as two bf16 terms: [hi (16) | lo (16)]
constexpr int kNout = 16;        // padded output width
constexpr int kMaxHidden = 4;
// SiLU layers run in base-2 units: their pre-activations u = -z log2(e)
// (input and biases scaled by -log2 e), their stored activations a/(-ln 2),
// absorbed by the next layer's weights (log2(e) ln 2 = 1) and the output
// layer's (scaled by -ln 2)
constexpr float kNegLog2e = -1.4426950408889634f, kNegLn2 = -0.6931471805599453f;
__host__ __device__ __forceinline__ float input_scale(int act) { return act == 0 ? kNegLog2e : 1.f; }
constexpr int kBiasCol = 13;     // X columns 13..15 (hi term) hold 1.0, against the bias terms
constexpr uint32_t kBiasTile = kWidth * 8 * 2;   // [128 x 8] bf16: columns 8..15 of a bias step's B
constexpr int kStashWords = 16;  // per-row pair data handed from builder to updater threads
// columns of a hidden layer's epilogue per TMEM read (16: four independent
// SiLU chains of a thread per wait; 32 spilled at the 128-register cap of a
// 512-thread CTA and measured slower, 2.57 against 2.51 ms per collide)
constexpr int kEpiW = 16;

template <int W>
__device__ __forceinline__ void tmem_ld_async(uint32_t taddr, uint32_t* r) {
  if (W == 32) tc::ld32_async(taddr, r);
  else tc::ld16_async(taddr, r);
}
template <int W>
__device__ __forceinline__ void tmem_wait_ld(uint32_t* r) {
  if (W == 32) tc::wait_ld32(r);
  else tc::wait_ld16(r);
}

// dynamic shared memory layout (bytes).  The weights are shared; each of the
// `slots` tile slots (one per warp group) has its own X, activation tiles,
// mbarrier and flag.
struct MlpLayout {
  uint32_t w_out, w_in, w_sq, w_zero, w_bias, slot0, slot_bytes, bias, ybuf, ybuf_bytes, mbar, tptr, flag, claim,
      fail, stash, total;
  int slots;
  __host__ __device__ uint32_t x(int g) const { return slot0 + (uint32_t)g * slot_bytes; }
};

constexpr uint32_t kMaxSmem = 232448 - 1024;  // 227 KB opt-in per CTA, less the static shared memory

__host__ __device__ inline MlpLayout mlp_layout(int n_hidden, int slots) {
  MlpLayout L;
  L.slots = slots;
  L.w_out = 0;                                        // FP32 [3 x 128] output layer
  L.w_in = L.w_out + 3 * kWidth * 4;                  // [128 x 32] = [W1 | W1]
  L.w_sq = L.w_in + kWidth * kKin * 2;                // (n_hidden-1) x [128 x 128]
  L.w_zero = L.w_sq + (uint32_t)(n_hidden - 1) * kWidth * kWidth * 2;   // [128 x 8] zeros
  L.w_bias = L.w_zero + kBiasTile;                   // (n_hidden-1) x [128 x 8] bias terms
  L.slot0 = L.w_bias + (uint32_t)(n_hidden - 1) * kBiasTile;
  L.slot_bytes = kTileM * kKin * 2;                  // X [128 x 32] (hi | lo)
  L.bias = L.slot0 + (uint32_t)slots * L.slot_bytes;  // floats: n_hidden*128 + 16
  // per slot: partial outputs of the column groups other than the first
  L.ybuf = L.bias + (uint32_t)(n_hidden * kWidth + kNout) * 4;
  L.ybuf_bytes = (uint32_t)(kThreads / slots / kTileM - 1) * kTileM * 3 * 4;
  L.mbar = L.ybuf + (uint32_t)slots * L.ybuf_bytes;
  L.mbar = (L.mbar + 15u) & ~15u;                     // slots x 8 bytes
  L.tptr = L.mbar + 16;
  L.flag = L.tptr + 4;                                // slots x 4 bytes: 1 until an MMA wait of the group times out
  L.claim = L.flag + 8;                               // slots x 4 bytes: next claimed unit
  L.fail = L.claim + 8;                               // slots x 4 bytes: a dependency wait failed
  // slots x 2 buffers x kStashWords x 128 words (word-major: a warp's rows
  // are consecutive words)
  L.stash = (L.fail + 8 + 15u) & ~15u;
  L.total = L.stash + (uint32_t)slots * 2 * kStashWords * kTileM * 4 + 256;
  return L;
}

// two tile slots (ping-pong warp groups) when they fit in shared memory
__host__ __device__ inline int mlp_slots(int n_hidden) {
  return mlp_layout(n_hidden, 2).total <= kMaxSmem ? 2 : 1;
}

struct MlpShape {
  int d_in, n_hidden, act, slots;
};

// bf16 bits of x, rounded to nearest even
__device__ __forceinline__ uint16_t bf16_bits(float x) { return (uint16_t)(tc::pack_bf16x2(x, 0.f) & 0xFFFFu); }

// A bias b as three bf16 terms b0 + b1 + b2 (b0 = bf16(b), b1 = bf16(b - b0),
// b2 = bf16(b - b0 - b1); the differences are exact in FP32): 24 significant
// bits, FP32's, so the MMA that multiplies them by 1.0 adds b to the
// accumulator up to its FP32 rounding.
__device__ __forceinline__ void bias_terms(float b, uint16_t r[3]) {
  r[0] = bf16_bits(b);
  const float d1 = b - __uint_as_float((uint32_t)r[0] << 16);
  r[1] = bf16_bits(d1);
  r[2] = bf16_bits(d1 - __uint_as_float((uint32_t)r[1] << 16));
}

// Copy the caller's row-major [out x in] bf16 layers into K-major core-matrix
// tiles (zero padded) and the biases into shared memory.  The biases enter
// through the MMAs, against the input tile's constant columns 13..15 (1.0):
// layer 0's as its weight columns 13..15, a hidden layer's in one more K
// step over the input tile's first 16 columns, issued first with the
// accumulator overwritten, whose B is zero in columns 0..12 and holds the
// bias terms in 13..15.  That B is two K-adjacent core-matrix columns: the
// first (columns 0..7) a zero tile shared by the layers, the second
// (columns 8..15) the layer's [128 x 8] bias tile, which the descriptor's
// K-direction offset reaches.
__device__ void load_weights(char* smem, const MlpLayout& L, const MlpShape& sh,
                             const uint16_t* __restrict__ w, const float* __restrict__ bias) {
  const int t = threadIdx.x, nt = blockDim.x;
  uint32_t* z = (uint32_t*)(smem + L.w_in);
  for (int q = t; q < (kWidth * kKin * 2) / 4; q += nt) z[q] = 0u;
  uint32_t* zb = (uint32_t*)(smem + L.w_zero);
  for (int q = t; q < (int)(sh.n_hidden * kBiasTile / 4); q += nt) zb[q] = 0u;
  __syncthreads();
  const float zs = input_scale(sh.act);
  for (int n = t; n < sh.n_hidden * kWidth; n += nt) {
    uint16_t r[3];
    bias_terms(bias[n] * zs, r);
    const int l = n / kWidth, nn = n % kWidth;
    for (int k = 0; k < 3; ++k) {
      if (l == 0)
        *(uint16_t*)(smem + L.w_in + tc::kmajor_offset(nn, kBiasCol + k, kKin)) = r[k];
      else
        *(uint16_t*)(smem + L.w_bias + (uint32_t)(l - 1) * kBiasTile + tc::kmajor_offset(nn, kBiasCol - 8 + k, 8)) =
            r[k];
    }
  }
  // layer 0: [128 x d_in], stored twice (columns k and 16 + k) so that the
  // two bf16 terms of the input share the weights
  for (int e = t; e < kWidth * sh.d_in; e += nt) {
    const int n = e / sh.d_in, k = e % sh.d_in;
    *(uint16_t*)(smem + L.w_in + tc::kmajor_offset(n, k, kKin)) = w[e];
    *(uint16_t*)(smem + L.w_in + tc::kmajor_offset(n, 16 + k, kKin)) = w[e];
  }
  const uint16_t* wl = w + kWidth * sh.d_in;
  for (int l = 0; l < sh.n_hidden - 1; ++l) {
    char* dst = smem + L.w_sq + (uint32_t)l * kWidth * kWidth * 2;
    for (int e = t; e < kWidth * kWidth; e += nt) {
      const int n = e >> 7, k = e & 127;
      *(uint16_t*)(dst + tc::kmajor_offset(n, k, kWidth)) = wl[e];
    }
    wl += kWidth * kWidth;
  }
  // output layer in FP32 [3 x 128] for the CUDA-core dot products
  float* wo = (float*)(smem + L.w_out);
  const float os = sh.act == 0 ? kNegLn2 : 1.f;
  for (int e = t; e < 3 * kWidth; e += nt) wo[e] = __uint_as_float((uint32_t)wl[e] << 16) * os;
  float* bs = (float*)(smem + L.bias);
  for (int e = t; e < sh.n_hidden * kWidth; e += nt) bs[e] = bias[e];
  for (int e = t; e < kNout; e += nt) bs[sh.n_hidden * kWidth + e] = e < 3 ? bias[sh.n_hidden * kWidth + e] : 0.f;
  tc::fence_async_smem();   // the operand tiles are read by the tensor core (async proxy)
}

__device__ __forceinline__ float act_f(int act, float z) {
  if (act == 1) return fmaxf(z, 0.f);
  return __fdividef(z, 1.f + __expf(-z));   // SiLU(z) = z / (1 + e^-z)
}

// The warp group a thread belongs to: G groups of blockDim/G threads, group g
// owning tile slot g, TMEM columns [128 g, 128 g + 128) and named barrier 1 + g.
struct Group {
  int g, G, t, nthr;  // group index, group count, thread index in the group, threads per group
};

__device__ __forceinline__ Group my_group(int G) {
  const int nthr = blockDim.x / G;
  return Group{(int)threadIdx.x / nthr, G, (int)threadIdx.x % nthr, nthr};
}

__device__ __forceinline__ void group_sync(const Group& q) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + q.g), "r"(q.nthr) : "memory");
}

// Run all layers on the X tile already in the group's slot (fenced and
// synchronised by the caller).  Returns false if a bounded wait ran out
// (status recorded); y receives the output row (+ bias) of group thread q.t
// for q.t < 128.  Rows: warp w of the group reads TMEM lanes 32 (w % 4) ..
// +31, i.e. row = 32 (w % 4) + lane; the columns of a hidden layer are split
// over the group's warps that share a lane group.  The hidden layers run on
// the tensor cores; the 3-wide output layer is a dot product on the CUDA
// cores inside the last hidden layer's epilogue (FP32 activations times the
// bf16 weights, summed in FP32), its column-group partials combined through
// shared memory -- no tensor-core pass, barrier and TMEM read for 3 outputs.
__device__ bool mlp_tile(char* smem, const MlpLayout& L, const MlpShape& sh, const Group& q,
                         uint32_t tmem, uint32_t& phase, float y[3], int* status, uint32_t xs) {
  // every layer's bias enters through its MMAs (the first one overwrites the
  // accumulator)
  const int gw = q.t >> 5;
  const int row = ((gw & 3) << 5) | (q.t & 31);
  const int cgroups = q.nthr / kTileM, cg = gw >> 2;
  const int cols = kWidth / cgroups;
  uint64_t* mbar = (uint64_t*)(smem + L.mbar) + q.g;
  volatile int* flag = (volatile int*)(smem + L.flag) + q.g;
  const uint32_t sbase = tc::smem_u32(smem);
  const uint32_t acc = tmem + (uint32_t)(q.g * 2 * kWidth);
  // the next layer's A operand: hi in columns [0, 64) of this region, lo in [64, 128)
  const uint32_t a_hi = acc + kWidth, a_lo = a_hi + kWidth / 2;
  const uint32_t lane_q = (uint32_t)((gw & 3) * 32) << 16;
  const uint32_t lane_tm = acc + lane_q;
  const float* bs = (const float*)(smem + L.bias);
  const float* wo = (const float*)(smem + L.w_out);
  // output-layer partial sums, even and odd columns apart
  float2 yq0 = make_float2(0.f, 0.f), yq1 = yq0, yq2 = yq0;
  for (int l = 0; l < sh.n_hidden; ++l) {
    if (q.t == 0) {
      tc::fence_after();
      if (l == 0) {
#pragma unroll
        for (int s = 0; s < kKin / 16; ++s)
          tc::mma_bf16(acc, tc::sdesc(sbase + xs + 256u * s, 128, kKin * 16),
                       tc::sdesc(sbase + L.w_in + 256u * s, 128, kKin * 16),
                       tc::idesc_bf16(kTileM, kWidth), s > 0);
      } else {
        const uint32_t wb = L.w_sq + (uint32_t)(l - 1) * kWidth * kWidth * 2;
        const uint32_t idesc = tc::idesc_bf16(kTileM, kWidth);
        // the bias: the input tile's first 16 columns (1.0 in 13..15) against
        // [zeros | the layer's bias tile] (core-matrix rows 128 bytes apart)
        tc::mma_bf16(acc, tc::sdesc(sbase + xs, 128, kKin * 16),
                     tc::sdesc(sbase + L.w_zero, L.w_bias + (uint32_t)(l - 1) * kBiasTile - L.w_zero, 128), idesc, 0);
        // activations enter as hi + lo bf16 terms against the same weights
#pragma unroll
        for (int s = 0; s < kWidth / 16; ++s)
          tc::mma_bf16_ta(acc, a_hi + 8u * s, tc::sdesc(sbase + wb + 256u * s, 128, 2048), idesc, 1);
#pragma unroll
        for (int s = 0; s < kWidth / 16; ++s)
          tc::mma_bf16_ta(acc, a_lo + 8u * s, tc::sdesc(sbase + wb + 256u * s, 128, 2048), idesc, 1);
      }
      tc::commit(mbar);
    }
    // every thread waits for the layer's MMAs itself (no barrier after the
    // issue); a timeout clears the group's flag, read after the group's next
    // barrier so that all its threads leave together
    if (!tc::mbar_wait(mbar, phase, status, kBarrierLimitNs)) *flag = 0;
    phase ^= 1u;
    tc::fence_after();
    const bool last = l == sh.n_hidden - 1;
    // this warp's columns in 16-wide pieces, the TMEM read of the next piece
    // in flight while the current one is processed
    const int cbeg = cg * cols, npieces = cols / kEpiW;
    uint32_t ra[kEpiW], rb[kEpiW];
    tmem_ld_async<kEpiW>(lane_tm + (uint32_t)cbeg, ra);
    tmem_wait_ld<kEpiW>(ra);
#pragma unroll 1
    for (int pc = 0; pc < npieces; pc += 2) {
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        if (pc + half >= npieces) break;
        uint32_t* cur = half ? rb : ra;
        uint32_t* nxt = half ? ra : rb;
        const int c0 = cbeg + kEpiW * (pc + half);
        const bool more = pc + half + 1 < npieces;
        if (more) tmem_ld_async<kEpiW>(lane_tm + (uint32_t)(c0 + kEpiW), nxt);
        // values in packed pairs (columns 2k, 2k + 1; the bias is already in
        // them): activation products, residuals and output-layer FMAs run two
        // per instruction
        float2 v[kEpiW / 2];
#pragma unroll
        for (int k = 0; k < kEpiW / 2; ++k)
          v[k] = make_float2(__uint_as_float(cur[2 * k]), __uint_as_float(cur[2 * k + 1]));
        if (sh.act == 0) {
#pragma unroll
          for (int k = 0; k < kEpiW / 2; k += 2) tc::silu2_4x2(v[k], v[k + 1]);
        } else {
#pragma unroll
          for (int k = 0; k < kEpiW / 2; ++k) v[k] = make_float2(act_f(sh.act, v[k].x), act_f(sh.act, v[k].y));
        }
        if (last) {
          const float2* w0 = (const float2*)(wo + c0);
          const float2* w1 = (const float2*)(wo + kWidth + c0);
          const float2* w2 = (const float2*)(wo + 2 * kWidth + c0);
#pragma unroll
          for (int k = 0; k < kEpiW / 2; ++k) {
            yq0 = __ffma2_rn(v[k], w0[k], yq0);
            yq1 = __ffma2_rn(v[k], w1[k], yq1);
            yq2 = __ffma2_rn(v[k], w2[k], yq2);
          }
        } else {
          uint32_t pk[kEpiW / 2], lo[kEpiW / 2];
          const float2 m1 = make_float2(-1.f, -1.f);
#pragma unroll
          for (int k = 0; k < kEpiW / 2; ++k) {
            pk[k] = tc::pack_bf16x2(v[k].x, v[k].y);
            // a - hi is exact (hi is a rounding of a); as an FMA with -1
            const float2 r = __ffma2_rn(make_float2(__uint_as_float(pk[k] << 16), __uint_as_float(pk[k] & 0xFFFF0000u)),
                                        m1, v[k]);
            lo[k] = tc::pack_bf16x2(r.x, r.y);
          }
          // columns c0 .. c0 + kEpiW - 1 of this row: kEpiW / 2 TMEM columns per term
#pragma unroll
          for (int h = 0; h < kEpiW / 16; ++h) {
            tc::st8_async(a_hi + lane_q + (uint32_t)((c0 >> 1) + 8 * h), pk + 8 * h);
            tc::st8_async(a_lo + lane_q + (uint32_t)((c0 >> 1) + 8 * h), lo + 8 * h);
          }
        }
        if (more) tmem_wait_ld<kEpiW>(nxt);
      }
    }
    // this thread's A operand stores complete before the next MMA
    if (!last) {
      tc::wait_st();
      tc::fence_before();
      group_sync(q);
      if (!*flag) return false;
    }
  }
  const float yp0 = yq0.x + yq0.y, yp1 = yq1.x + yq1.y, yp2 = yq2.x + yq2.y;
  // combine the column groups' partial outputs (column group 0 = the updaters)
  float* yb = (float*)(smem + L.ybuf + (uint32_t)q.g * L.ybuf_bytes);
  if (cg > 0) {
    float* d = yb + ((cg - 1) * kTileM + row) * 3;
    d[0] = yp0; d[1] = yp1; d[2] = yp2;
  }
  tc::fence_before();
  group_sync(q);
  if (!*flag) return false;
  if (cg == 0) {
    const float* bo = bs + sh.n_hidden * kWidth;
    float s0 = yp0, s1 = yp1, s2 = yp2;
    for (int g2 = 1; g2 < cgroups; ++g2) {
      const float* d = yb + ((g2 - 1) * kTileM + row) * 3;
      s0 += d[0]; s1 += d[1]; s2 += d[2];
    }
    y[0] = s0 + bo[0];
    y[1] = s1 + bo[1];
    y[2] = s2 + bo[2];
  }
  return true;
}

// Write row t of the X tile from 16 FP32 features (padding zeros included),
// x = scale * feature (the first layer's input scale): columns 0..15 hold
// hi = bf16(x), columns 16..31 lo = bf16(x - hi), so the first layer sees x
// to about 16 significant bits through bf16 operands.
// Columns 13..15 of hi hold 1.0 (and those of lo 0): against the weight
// columns that carry layer 0's bias terms.  Features occupy at most columns
// 0..7.
__device__ __forceinline__ void write_x_row(char* smem, uint32_t xoff, int t, const float* f, float scale) {
  const uint32_t sb = tc::smem_u32(smem) + xoff;
  uint32_t hi[8], lo[8];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const float x0 = f[2 * q] * scale, x1 = f[2 * q + 1] * scale;
    hi[q] = tc::pack_bf16x2(x0, x1);
    const float h0 = __uint_as_float(hi[q] << 16), h1 = __uint_as_float(hi[q] & 0xFFFF0000u);
    lo[q] = tc::pack_bf16x2(x0 - h0, x1 - h1);
  }
  static_assert(kBiasCol == 13, "the constant columns are 13, 14, 15");
  hi[6] = 0x3F800000u; hi[7] = 0x3F803F80u;   // columns 12 = 0, 13..15 = 1.0
  lo[6] = 0u; lo[7] = 0u;
  tc::st_shared_v4(sb + tc::kmajor_offset(t, 0, kKin), hi[0], hi[1], hi[2], hi[3]);
  tc::st_shared_v4(sb + tc::kmajor_offset(t, 8, kKin), hi[4], hi[5], hi[6], hi[7]);
  tc::st_shared_v4(sb + tc::kmajor_offset(t, 16, kKin), lo[0], lo[1], lo[2], lo[3]);
  tc::st_shared_v4(sb + tc::kmajor_offset(t, 24, kKin), lo[4], lo[5], lo[6], lo[7]);
}

// CTA prologue/epilogue: TMEM allocation by warp 0 (per tile slot 128
// accumulator columns and 128 columns of A operand), one mbarrier per slot.
__device__ __forceinline__ uint32_t tmem_cols(int slots) { return slots > 1 ? 512u : 256u; }

__device__ __forceinline__ uint32_t cta_setup(char* smem, const MlpLayout& L) {
  if (threadIdx.x < 32) {
    tc::tmem_alloc((uint32_t*)(smem + L.tptr), tmem_cols(L.slots));
    tc::tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    for (int g = 0; g < L.slots; ++g) {
      tc::mbar_init((uint64_t*)(smem + L.mbar) + g, 1);
      ((volatile int*)(smem + L.flag))[g] = 1;   // the group's MMA waits have not failed
    }
    tc::mbar_fence_init();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  return *(volatile uint32_t*)(smem + L.tptr);
}

__device__ __forceinline__ void cta_teardown(uint32_t tmem, const MlpLayout& L) {
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (threadIdx.x < 32) tc::tmem_dealloc(tmem, tmem_cols(L.slots));
}

// ---------------------------------------------------------------- standalone forward
// y[n x 3] = f_theta(x[n x d_in]) on bf16 tensor cores.
__global__ void __launch_bounds__(kThreads) k_mlp_forward(MlpShape sh, const uint16_t* __restrict__ w,
                                                        const float* __restrict__ bias, int64_t n,
                                                        const float* __restrict__ x, float* __restrict__ y,
                                                        int* status) {
  extern __shared__ __align__(1024) char smem[];
  const MlpLayout L = mlp_layout(sh.n_hidden, sh.slots);
  load_weights(smem, L, sh, w, bias);
  const uint32_t tmem = cta_setup(smem, L);
  const Group q = my_group(L.slots);
  uint32_t phase = 0;
  const int64_t tiles = (n + kTileM - 1) / kTileM;
  for (int64_t tile = blockIdx.x + (int64_t)gridDim.x * q.g; tile < tiles; tile += (int64_t)gridDim.x * q.G) {
    const int64_t row = tile * kTileM + q.t;
    if (q.t < kTileM) {
      float f[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) f[k] = 0.f;
      if (row < n)
        for (int k = 0; k < sh.d_in; ++k) f[k] = x[row * sh.d_in + k];
      write_x_row(smem, L.x(q.g), q.t, f, input_scale(sh.act));
      tc::fence_async_smem();
    }
    group_sync(q);
    float o[3];
    if (!mlp_tile(smem, L, sh, q, tmem, phase, o, status, L.x(q.g))) break;   // status recorded
    if (q.t < kTileM && row < n) { y[3 * row] = o[0]; y[3 * row + 1] = o[1]; y[3 * row + 2] = o[2]; }
  }
  cta_teardown(tmem, L);
}

// ---------------------------------------------------------------- tensor-core self test
// D[128 x N] = A[128 x K] B[N x K]^T with the same operand layout and MMA
// issue as the MLP (one CTA).  layout bit 0: A stored MN-major (the tile of
// A^T, rows = k), bit 1: B stored MN-major, bit 2: exchange the roles of the
// two descriptor offsets for MN-major operands (diagnostic), bit 3: A in
// tensor memory (row m in lane m, columns 256 + k/2, two bf16 per column).
__device__ __forceinline__ uint64_t operand_desc(uint32_t base, int mn_major, int swap, int MN, int K, int s) {
  if (!mn_major) return tc::sdesc(base + 256u * s, 128, (uint32_t)(K / 8) * 128);
  // MN-major: core matrices along MN are 128 B apart, along K (8 rows) MN/8*128 B
  const uint32_t mn_stride = 128, k_stride = (uint32_t)(MN / 8) * 128;
  const uint32_t start = base + 2u * k_stride * s;
  return swap ? tc::sdesc(start, mn_stride, k_stride) : tc::sdesc(start, k_stride, mn_stride);
}

__global__ void __launch_bounds__(128) k_tc_selftest(int N, int K, int layout, const uint16_t* __restrict__ A,
                                                     const uint16_t* __restrict__ B, float* __restrict__ D,
                                                     int* status) {
  extern __shared__ __align__(1024) char smem[];
  const uint32_t a_off = 0, b_off = 128u * K * 2, mb = b_off + (uint32_t)N * K * 2;
  const uint32_t tp = mb + 8, fl = tp + 4;
  const int t = threadIdx.x;
  const int a_mn = layout & 1, b_mn = (layout >> 1) & 1, swap = (layout >> 2) & 1, a_tm = (layout >> 3) & 1;
  for (int e = t; e < 128 * K && !a_tm; e += 128) {
    const int m = e / K, k = e % K;
    *(uint16_t*)(smem + a_off + (a_mn ? tc::kmajor_offset(k, m, 128) : tc::kmajor_offset(m, k, K))) = A[e];
  }
  for (int e = t; e < N * K; e += 128) {
    const int n = e / K, k = e % K;
    *(uint16_t*)(smem + b_off + (b_mn ? tc::kmajor_offset(k, n, N) : tc::kmajor_offset(n, k, K))) = B[e];
  }
  uint32_t ncols = 32;
  while ((int)ncols < N) ncols <<= 1;
  if (a_tm) ncols = 512;   // D in columns [0, N), A in [256, 256 + K/2)
  if (t < 32) { tc::tmem_alloc((uint32_t*)(smem + tp), ncols); tc::tmem_relinquish(); }
  if (t == 0) { tc::mbar_init((uint64_t*)(smem + mb), 1); tc::mbar_fence_init(); }
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *(volatile uint32_t*)(smem + tp);
  const uint32_t sbase = tc::smem_u32(smem);
  volatile int* flag = (volatile int*)(smem + fl);
  if (a_tm) {
    // row t of A into lane t: columns 256 + k/2, k even in the low half
    const uint32_t lane_a = tmem + ((uint32_t)((t >> 5) * 32) << 16) + 256u;
    for (int c0 = 0; c0 < K / 2; c0 += 8) {
      uint32_t r[8];
      for (int q = 0; q < 8; ++q)
        r[q] = (uint32_t)A[t * K + 2 * (c0 + q)] | ((uint32_t)A[t * K + 2 * (c0 + q) + 1] << 16);
      tc::st8_async(lane_a + (uint32_t)c0, r);
    }
    tc::wait_st();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
  }
  if (t == 0) {
    const uint32_t idesc = tc::idesc_bf16(128, N) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16);
    for (int s = 0; s < K / 16; ++s) {
      if (a_tm)
        tc::mma_bf16_ta(tmem, tmem + 256u + 8u * s, operand_desc(sbase + b_off, b_mn, swap, N, K, s), idesc, s > 0);
      else
        tc::mma_bf16(tmem, operand_desc(sbase + a_off, a_mn, swap, 128, K, s),
                     operand_desc(sbase + b_off, b_mn, swap, N, K, s), idesc, s > 0);
    }
    tc::commit((uint64_t*)(smem + mb));
    *flag = tc::mbar_wait((uint64_t*)(smem + mb), 0, status, kBarrierLimitNs) ? 1 : 0;
  }
  __syncthreads();
  tc::fence_after();
  if (*flag) {
    const uint32_t lane_tm = tmem + ((uint32_t)((t >> 5) * 32) << 16);
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      tc::ld16(lane_tm + (uint32_t)c0, v);
      for (int q = 0; q < 16; ++q) D[t * N + c0 + q] = v[q];
    }
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (t < 32) tc::tmem_dealloc(tmem, ncols);
}

// ---------------------------------------------------------------- collide
struct NeuralArgs {
  uint64_t seed, step;
  const uint64_t* step_dev;
  double sigma_v_inv, T_ref_inv, m_over_3k, eps;
  float sigma_v_inv_f, T_feat_f;  // 1/sigma_v and m/(3 k T_ref) in FP32 for the MLP inputs
  const double* mom;
  float* u_out;
  const int4* pairs;
  const uint32_t* deps;
  const int32_t* ro;
  const dsmc_select_info_t* info;
  double *vx, *vy, *vz;
  unsigned* done;
  unsigned* bar;   // [2] abort word, [3] unit cursor
  int* status;
};

// Box-Muller pair in FP32 from the top 24 bits of two Philox words:
// rho = sqrt(-2 ln(1 - U1)), theta = 2 pi U2 (U1, U2 in [0, 1)).  The MLP
// sees the normals through bf16 terms, far coarser than FP32.
__device__ __forceinline__ void box_muller_f(uint32_t w1, uint32_t w2, float* z0, float* z1) {
  const float u1 = (float)(w1 >> 8) * 5.9604645e-8f, u2 = (float)(w2 >> 8) * 5.9604645e-8f;
  const float rho = sqrtf(-2.f * __logf(1.f - u1));
  float s, c;
  __sincosf(6.2831853f * u2, &s, &c);
  *z0 = rho * c;
  *z1 = rho * s;
}

// Build the MLP input row of pair p (features in FP32, Sec. 2.2 Eq. (mlp_input))
// into the group's X tile and stash what the pair update needs -- p, the
// particle slots and the six velocity components -- in word w of the row at
// stash[w * 128 + row] (shared memory).  p < 0 marks a padding row.
__device__ __forceinline__ void build_row(char* smem, uint32_t xoff, volatile int* fail, const MlpShape& sh,
                                          const NeuralArgs& a, int row, int32_t p, uint32_t* stash) {
  float f[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) f[c] = 0.f;
  uint32_t st[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) st[c] = 0u;
  st[0] = (uint32_t)-1;
  int4 q = make_int4(0, 0, 0, 0);
  if (p >= 0) {
    q = a.pairs[p];
    // the previous pairs of both particles must be done (bounded wait)
    if (!wait_deps(a.done, q.x, q.y, a.deps[p], a.bar + 2, a.status)) {
      *fail = 1;
      p = -1;
    }
  }
  // the lanes leave their waits at different times: the gather, the draws
  // and the input row run with the warp reconverged
  __syncwarp();
  if (p >= 0) {
    const double xi = __ldcg(a.vx + q.x), yi = __ldcg(a.vy + q.x), zi = __ldcg(a.vz + q.x);
    const double xj = __ldcg(a.vx + q.y), yj = __ldcg(a.vy + q.y), zj = __ldcg(a.vz + q.y);
    // MLP inputs need FP32 only: convert on the integer pipe, subtract and
    // scale in FP32 (error ~ |v| 2^-24, far below the bf16 input terms)
    f[0] = (f64_to_f32(xi) - f64_to_f32(xj)) * a.sigma_v_inv_f;
    f[1] = (f64_to_f32(yi) - f64_to_f32(yj)) * a.sigma_v_inv_f;
    f[2] = (f64_to_f32(zi) - f64_to_f32(zj)) * a.sigma_v_inv_f;
    const u32x4 wa = draw(a.seed, (uint32_t)q.w, (uint32_t)q.z, a.step, TAG_NOISE, 0);
    const u32x4 wb = draw(a.seed, (uint32_t)q.w, (uint32_t)q.z, a.step, TAG_NOISE, 1);
    float z[4];
    box_muller_f(wa.x, wa.z, &z[0], &z[1]);
    box_muller_f(wb.x, wb.z, &z[2], &z[3]);
    if (sh.d_in == 8) {
      const double* m = a.mom + 5 * (size_t)q.z;
      f[3] = f64_to_f32(m[4]) / f64_to_f32(m[0]) * a.T_feat_f;
      f[4] = z[0]; f[5] = z[1]; f[6] = z[2]; f[7] = z[3];
    } else {
      f[3] = z[0]; f[4] = z[1]; f[5] = z[2];
    }
    st[0] = (uint32_t)p; st[1] = (uint32_t)q.x; st[2] = (uint32_t)q.y;
    const double v[6] = {xi, yi, zi, xj, yj, zj};
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      st[4 + 2 * c] = __double2loint(v[c]);
      st[5 + 2 * c] = __double2hiint(v[c]);
    }
  }
  write_x_row(smem, xoff, row, f, input_scale(sh.act));
  tc::fence_async_smem();
#pragma unroll
  for (int c = 0; c < kStashWords; ++c) stash[c * kTileM + row] = st[c];
}

// Pair update of one row from the MLP output y and the row's stash:
// shell projection v_r' = |v_r| y/|y| and centre-of-mass update in FP64.
// s = |v_r|/|y| from an FP32 estimate and one FP64 Newton step on
// s^2 |y|^2 = |v_r|^2 (relative error ~1e-14), so |v_r'| = |v_r|.
__device__ __forceinline__ void update_row(const NeuralArgs& a, const float y[3], const uint32_t* stash,
                                           int row, unsigned round1) {
  uint32_t st[16];
#pragma unroll
  for (int c = 0; c < kStashWords; ++c) st[c] = stash[c * kTileM + row];
  const int32_t p = (int32_t)st[0];
  if (p < 0) return;
  const int32_t qi = (int32_t)st[1], qj = (int32_t)st[2];
  double v[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) v[c] = __hiloint2double((int)st[5 + 2 * c], (int)st[4 + 2 * c]);
  const double ux = v[0] - v[3], uy = v[1] - v[4], uz = v[2] - v[5];
  const double g2 = ux * ux + uy * uy + uz * uz;
  // the FP32 <-> FP64 conversions on the integer pipe (GB300's FP64 pipe,
  // which runs the conversion instructions, bounds this update)
  double y0 = f32_to_f64(y[0]), y1 = f32_to_f64(y[1]), y2 = f32_to_f64(y[2]);
  const double ny2 = y0 * y0 + y1 * y1 + y2 * y2;
  const float g2f = f64_to_f32(g2);
  // (a pair with g = 0, or g^2 below the FP32 range, takes the other branch:
  // v_r' = g e = 0 up to ~1e-19 m/s, where the shell scale would divide by 0)
  if (ny2 > a.eps * a.eps && g2f > 0.f) {
    const float ny2f = f64_to_f32(ny2);
    const float sf = sqrtf(g2f / ny2f);
    const double s0 = f32_to_f64(sf);
    const double res = g2 - s0 * s0 * ny2;           // g2 - s0^2 ny2
    const double sc = s0 + res * f32_to_f64(0.5f * sf / g2f);
    y0 *= sc; y1 *= sc; y2 *= sc;                    // v_r'
  } else {  // isotropic fallback direction (tag 3)
    const int4 q = a.pairs[p];
    const u32x4 wi = draw(a.seed, (uint32_t)q.w, (uint32_t)q.z, a.step, TAG_ISO);
    const double c = 2.0 * u53(wi.x, wi.y) - 1.0, sn = sqrt(1.0 - c * c);
    double se, ce;
    sincos(2.0 * DSMC_PI * u53(wi.z, wi.w), &se, &ce);
    const double g = sqrt(g2);
    y0 = g * c; y1 = g * sn * ce; y2 = g * sn * se;
  }
  if (a.u_out) {
    const double ig = g2 > 0.0 ? 1.0 / sqrt(g2) : 0.0;
    a.u_out[3 * (size_t)p] = (float)(y0 * ig); a.u_out[3 * (size_t)p + 1] = (float)(y1 * ig);
    a.u_out[3 * (size_t)p + 2] = (float)(y2 * ig);
  }
  const double cx = 0.5 * (v[0] + v[3]), cy = 0.5 * (v[1] + v[4]), cz = 0.5 * (v[2] + v[5]);
  __stcg(a.vx + qi, fma(0.5, y0, cx)); __stcg(a.vy + qi, fma(0.5, y1, cy)); __stcg(a.vz + qi, fma(0.5, y2, cz));
  __stcg(a.vx + qj, fma(-0.5, y0, cx)); __stcg(a.vy + qj, fma(-0.5, y1, cy)); __stcg(a.vz + qj, fma(-0.5, y2, cz));
  release_pair(a.done, qi, qj, round1);
}

// ---------------------------------------------------------------- pipelined collide
// A CTA of 768 threads: two MLP warp groups of 8 warps (threads 0..511, TMEM
// columns and tile work as in mlp_tile), four builder warps (512..639) and
// four updater warps (640..767).  Tiles of 128 pairs of one round are
// claimed by the builders from a global cursor in round-major order and
// handed to the two MLP groups alternately through three buffers per group
// (the input tile X, the per-row pair data the update needs, the MLP output
// y, the tile's pair range and round): builders build tile k + 2 (waiting,
// bounded, until the previous pairs of its particles are done) while an MLP
// group runs the layers of tile k + 1 and the updaters apply the pair updates
// of tile k and stamp its particles done.  So the MLP groups never wait for
// the latency-bound build or the FP64 update.  Hand-offs are mbarriers:
// built (128 builder arrivals), ydone (the 128 threads that hold y), freed
// (128 updater arrivals); each buffer is reused every third tile of its
// group.  No wait can be circular: a build only waits on tiles claimed
// earlier, whose MLP and update stages never wait on a later build.  Every
// wait is bounded and ends early once any role of the CTA (or a dependency
// wait of any CTA) has failed.
constexpr int kPipeThreads = 768;
constexpr int kPipeBufs = 3;
constexpr int kBuildBase = 512, kUpdateBase = 640, kRoleThreads = 128;

struct PipeLayout {
  MlpLayout m;        // weights, biases, per-group MMA barriers, TMEM pointer, column-group partials
  uint32_t x0, st0, y0, info0, bars, abort, bcast, total;
  __host__ __device__ uint32_t buf(int g, int b) const { return (uint32_t)(g * kPipeBufs + b); }
  __host__ __device__ uint32_t x(int g, int b) const { return x0 + buf(g, b) * (uint32_t)(kTileM * kKin * 2); }
  __host__ __device__ uint32_t st(int g, int b) const { return st0 + buf(g, b) * (uint32_t)(kStashWords * kTileM * 4); }
  __host__ __device__ uint32_t y(int g, int b) const { return y0 + buf(g, b) * (uint32_t)(kTileM * 3 * 4); }
  __host__ __device__ uint32_t info(int g, int b) const { return info0 + buf(g, b) * 16u; }
  // mbarriers: built[6], ydone[6], freed[6]
  __host__ __device__ uint32_t built(int g, int b) const { return bars + buf(g, b) * 8u; }
  __host__ __device__ uint32_t ydone(int g, int b) const { return bars + (6u + buf(g, b)) * 8u; }
  __host__ __device__ uint32_t freed(int g, int b) const { return bars + (12u + buf(g, b)) * 8u; }
};

__host__ __device__ inline PipeLayout pipe_layout(int n_hidden) {
  PipeLayout P;
  MlpLayout& L = P.m;
  L.slots = 2;
  L.w_out = 0;
  L.w_in = L.w_out + 3 * kWidth * 4;
  L.w_sq = L.w_in + kWidth * kKin * 2;
  L.w_zero = L.w_sq + (uint32_t)(n_hidden - 1) * kWidth * kWidth * 2;
  L.w_bias = L.w_zero + kBiasTile;
  L.slot0 = 0;                                   // (the X tiles are per buffer below)
  L.slot_bytes = 0;
  L.bias = L.w_bias + (uint32_t)(n_hidden - 1) * kBiasTile;
  L.ybuf = L.bias + (uint32_t)(n_hidden * kWidth + kNout) * 4;
  L.ybuf_bytes = (uint32_t)(256 / kTileM - 1) * kTileM * 3 * 4;   // 8-warp groups: 2 column groups
  L.mbar = (L.ybuf + 2 * L.ybuf_bytes + 15u) & ~15u;
  L.tptr = L.mbar + 16;
  L.flag = L.tptr + 4;
  L.claim = L.flag + 8;
  L.fail = L.claim + 8;
  L.stash = 0;
  P.x0 = (L.fail + 8 + 127u) & ~127u;            // X tiles: K-major core matrices
  P.st0 = P.x0 + 2 * kPipeBufs * kTileM * kKin * 2;
  P.y0 = P.st0 + 2 * kPipeBufs * kStashWords * kTileM * 4;
  P.info0 = P.y0 + 2 * kPipeBufs * kTileM * 3 * 4;
  P.bars = (P.info0 + 2 * kPipeBufs * 16 + 7u) & ~7u;
  P.abort = P.bars + 18 * 8;
  P.bcast = P.abort + 16;
  P.total = P.bcast + 16 + 256;
  L.total = P.total;
  return P;
}

__device__ __forceinline__ bool pipe_aborted(char* smem, const PipeLayout& P, const NeuralArgs& a) {
  return *(volatile int*)(smem + P.abort) != 0 || ld_relaxed(a.bar + 2) != 0;
}
__device__ __forceinline__ void pipe_abort(char* smem, const PipeLayout& P, const NeuralArgs& a) {
  *(volatile int*)(smem + P.abort) = 1;
  atomicExch(a.bar + 2, 1u);
}

// Bounded wait for phase `parity` of an mbarrier, ending early once the CTA
// or the grid has aborted; false on timeout or abort (a timeout records
// DSMC_ERR_TIMEOUT and aborts).
__device__ __forceinline__ bool pipe_wait(char* smem, const PipeLayout& P, const NeuralArgs& a, uint32_t bar_off,
                                          uint32_t parity) {
  uint64_t* mb = (uint64_t*)(smem + bar_off);
  if (tc::mbar_try_wait(mb, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (;;) {
    if (tc::mbar_try_wait_hint(mb, parity, 2000u)) return true;
    if (pipe_aborted(smem, P, a)) return false;
    if (globaltimer_ns() - t0 > kBarrierLimitNs) {
      set_status(a.status, DSMC_ERR_TIMEOUT);
      pipe_abort(smem, P, a);
      return false;
    }
  }
}

__device__ __forceinline__ void mbar_arrive(char* smem, uint32_t bar_off) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(smem + bar_off)) : "memory");
}

// AND of a predicate over the `n` threads of named barrier `id`
__device__ __forceinline__ bool role_all(int id, int n, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
      "barrier.red.and.pred q, %2, %3, p;\n\tselp.u32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)pred), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void role_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }

__global__ void __launch_bounds__(kPipeThreads, 1) k_collide_neural(MlpShape sh, const uint16_t* __restrict__ w,
                                                                 const float* __restrict__ bias, NeuralArgs a) {
  if (a.step_dev) a.step = *a.step_dev;
  extern __shared__ __align__(1024) char smem[];
  const PipeLayout P = pipe_layout(sh.n_hidden);
  const MlpLayout& L = P.m;
  load_weights(smem, L, sh, w, bias);
  if (threadIdx.x == 0) {
    for (int q = 0; q < 6; ++q) {
      tc::mbar_init((uint64_t*)(smem + P.bars) + q, kRoleThreads);        // built
      tc::mbar_init((uint64_t*)(smem + P.bars) + 6 + q, kRoleThreads);    // ydone
      tc::mbar_init((uint64_t*)(smem + P.bars) + 12 + q, kRoleThreads);   // freed
    }
    *(volatile int*)(smem + P.abort) = 0;
  }
  const uint32_t tmem = cta_setup(smem, L);   // TMEM (512 columns), per-group MMA barriers; CTA-wide barrier
  const int R = a.info->n_rounds;
  const int t = threadIdx.x;
  if (t < kBuildBase) {
    // ------------------------------------------------ MLP groups
    const Group q{t / 256, 2, t % 256, 256};
    uint32_t phase = 0;
    const int row = (((q.t >> 5) & 3) << 5) | (q.t & 31);
    const bool yrow = q.t < kTileM;   // column group 0: holds the row's output
    for (int kk = 0;; ++kk) {
      const int b = kk % kPipeBufs;
      const bool ok = role_all(1 + q.g, 256, pipe_wait(smem, P, a, P.built(q.g, b), (uint32_t)(kk / kPipeBufs) & 1u));
      if (!ok) break;
      tc::fence_after();
      const int end = ((volatile int*)(smem + P.info(q.g, b)))[3];
      if (end) {
        if (yrow) mbar_arrive(smem, P.ydone(q.g, b));
        break;
      }
      float y[3];
      if (!mlp_tile(smem, L, sh, q, tmem, phase, y, a.status, P.x(q.g, b))) {
        pipe_abort(smem, P, a);
        break;
      }
      if (yrow) {
        float* yb = (float*)(smem + P.y(q.g, b)) + 3 * row;
        yb[0] = y[0]; yb[1] = y[1]; yb[2] = y[2];
        mbar_arrive(smem, P.ydone(q.g, b));
      }
    }
  } else if (t < kUpdateBase) {
    // ------------------------------------------------ builders
    const int tb = t - kBuildBase;
    int r = 0;
    int64_t base = 0;
    volatile int* fail = (volatile int*)(smem + P.abort);
    for (int k = 0;; ++k) {
      const int g = k & 1, kk = k >> 1, b = kk % kPipeBufs;
      bool ok = true;
      if (kk >= kPipeBufs) ok = pipe_wait(smem, P, a, P.freed(g, b), (uint32_t)(kk / kPipeBufs - 1) & 1u);
      if (!role_all(3, kRoleThreads, ok)) break;
      volatile unsigned* bc = (volatile unsigned*)(smem + P.bcast) + (k & 1);
      if (tb == 0) *bc = atomicAdd(a.bar + 3, 1u);
      role_sync(3, kRoleThreads);
      int32_t p0 = 0, p1 = 0;
      const bool have = unit_range(a.ro, R, kTileM, r, base, *bc, &p0, &p1);
      int* info = (int*)(smem + P.info(g, b));
      if (tb == 0) { info[0] = p0; info[1] = p1; info[2] = r; info[3] = have ? 0 : 1; }
      if (have) {
        const int32_t p = p0 + tb;
        build_row(smem, P.x(g, b), fail, sh, a, tb, p < p1 ? p : -1, (uint32_t*)(smem + P.st(g, b)));
      }
      mbar_arrive(smem, P.built(g, b));
      if (!have) {
        // the other group's next buffer carries the end too
        const int k2 = k + 1, g2 = k2 & 1, kk2 = k2 >> 1, b2 = kk2 % kPipeBufs;
        bool ok2 = true;
        if (kk2 >= kPipeBufs) ok2 = pipe_wait(smem, P, a, P.freed(g2, b2), (uint32_t)(kk2 / kPipeBufs - 1) & 1u);
        if (role_all(3, kRoleThreads, ok2)) {
          if (tb == 0) ((volatile int*)(smem + P.info(g2, b2)))[3] = 1;
          mbar_arrive(smem, P.built(g2, b2));
        }
        break;
      }
      if (*fail) pipe_abort(smem, P, a);
    }
  } else {
    // ------------------------------------------------ updaters
    const int tu = t - kUpdateBase;
    for (int k = 0;; ++k) {
      const int g = k & 1, kk = k >> 1, b = kk % kPipeBufs;
      if (!role_all(4, kRoleThreads, pipe_wait(smem, P, a, P.ydone(g, b), (uint32_t)(kk / kPipeBufs) & 1u))) break;
      const int* info = (const int*)(smem + P.info(g, b));
      if (((volatile const int*)info)[3]) break;
      const float* yb = (const float*)(smem + P.y(g, b)) + 3 * tu;
      const float y[3] = {yb[0], yb[1], yb[2]};
      update_row(a, y, (const uint32_t*)(smem + P.st(g, b)), tu, (unsigned)(info[2] + 1));
      mbar_arrive(smem, P.freed(g, b));
    }
  }
  cta_teardown(tmem, L);
}

// Failure-detection self test: wait on an mbarrier that no MMA commit will
// ever complete; the bounded wait must record DSMC_ERR_TIMEOUT and return.
__global__ void k_selftest_mbar(int* status, uint64_t limit_ns) {
  __shared__ __align__(8) uint64_t mbar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&mbar, 1);
    tc::mbar_fence_init();
    tc::mbar_wait(&mbar, 0, status, limit_ns);
  }
}

int launch_selftest_mbar(Ctx* c, uint64_t limit_ns, cudaStream_t s) {
  k_selftest_mbar<<<1, 32, 0, s>>>(status_ptr(c), limit_ns);
  count_launches(c, 1);
  return cudaGetLastError() == cudaSuccess ? 0 : DSMC_ERR_CUDA;
}


static bool set_smem(const void* k, int bytes) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess;
}

int launch_collide_neural(Ctx* c, const dsmc_gas_t& gas, const dsmc_mlp_t& mlp,
                          const uint16_t* w, const float* bias, uint64_t step,
                          const double* mom, int32_t n, const int32_t* pairs, const uint32_t* deps,
                          const int32_t* ro, const dsmc_select_info_t* info, double* vx, double* vy,
                          double* vz, float* u_out, void* ws, size_t ws_bytes, cudaStream_t s) {
  if (mlp.n_hidden > kMaxHidden) return record(c, DSMC_ERR_UNSUPPORTED, "collide_neural: n_hidden > 4");
  if (ws_bytes < collide_ws(n)) return record(c, DSMC_ERR_ARG, "collide_neural: workspace too small");
  const MlpShape sh{mlp.d_in, mlp.n_hidden, mlp.act, 2};
  const PipeLayout P = pipe_layout(sh.n_hidden);
  if (P.total > kMaxSmem) return record(c, DSMC_ERR_UNSUPPORTED, "collide_neural: layout exceeds shared memory");
  if (!set_smem((const void*)k_collide_neural, (int)P.total))
    return record(c, DSMC_ERR_CUDA, "collide_neural: shared-memory attribute");
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k_collide_neural, kPipeThreads, P.total) !=
          cudaSuccess || per_sm < 1)
    return record(c, DSMC_ERR_CUDA, "collide_neural: occupancy query failed");
  NeuralArgs a;
  a.seed = gas.seed; a.step = step; a.step_dev = graph_step_ptr(c);
  a.sigma_v_inv = 1.0 / mlp.sigma_v; a.T_ref_inv = 1.0 / mlp.T_ref;
  a.m_over_3k = gas.mass / (3.0 * DSMC_KB); a.eps = mlp.eps;
  a.sigma_v_inv_f = (float)a.sigma_v_inv;
  a.T_feat_f = (float)(a.m_over_3k * a.T_ref_inv);
  a.mom = mom; a.u_out = u_out; a.pairs = (const int4*)pairs; a.deps = deps; a.ro = ro; a.info = info;
  a.vx = vx; a.vy = vy; a.vz = vz; a.done = (unsigned*)ws; a.bar = barrier_ptr(c); a.status = status_ptr(c);
  if (cudaMemsetAsync(a.bar, 0, 4 * sizeof(unsigned), s) != cudaSuccess ||
      cudaMemsetAsync(a.done, 0, sizeof(unsigned) * (size_t)(n > 0 ? n : 1), s) != cudaSuccess)
    return DSMC_ERR_CUDA;
  k_collide_neural<<<sm_count(c) * per_sm, kPipeThreads, P.total, s>>>(sh, w, bias, a);
  count_launches(c, 1);
  return cudaGetLastError() == cudaSuccess ? 0 : record(c, DSMC_ERR_CUDA, "collide_neural: launch failed");
}

int launch_mlp_forward(Ctx* c, const dsmc_mlp_t& mlp, const uint16_t* w, const float* bias,
                       int64_t n, const float* x, float* y, cudaStream_t s) {
  if (n == 0) return 0;
  if (mlp.n_hidden > kMaxHidden) return record(c, DSMC_ERR_UNSUPPORTED, "mlp_forward: n_hidden > 4");
  const MlpShape sh{mlp.d_in, mlp.n_hidden, mlp.act, mlp_slots(mlp.n_hidden)};
  const MlpLayout L = mlp_layout(sh.n_hidden, sh.slots);
  if (!set_smem((const void*)k_mlp_forward, (int)L.total))
    return record(c, DSMC_ERR_CUDA, "mlp_forward: shared-memory attribute");
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k_mlp_forward, kThreads, L.total);
  if (per_sm < 1) per_sm = 1;
  const int64_t tiles = (n + kTileM - 1) / kTileM;
  int64_t blocks = (int64_t)sm_count(c) * per_sm;
  if (blocks > tiles) blocks = tiles;
  k_mlp_forward<<<(unsigned)blocks, kThreads, L.total, s>>>(sh, w, bias, n, x, y, status_ptr(c));
  count_launches(c, 1);
  return cudaGetLastError() == cudaSuccess ? 0 : DSMC_ERR_CUDA;
}

int launch_tc_selftest(Ctx* c, int N, int K, int layout, const uint16_t* A, const uint16_t* B, float* D,
                       cudaStream_t s) {
  // generous allocation: every reading of the descriptor offsets stays inside it
  const int smem = 200 * 1024;
  if (!set_smem((const void*)k_tc_selftest, smem)) return record(c, DSMC_ERR_CUDA, "tc_selftest: smem");
  k_tc_selftest<<<1, 128, smem, s>>>(N, K, layout, A, B, D, status_ptr(c));
  count_launches(c, 1);
  return cudaGetLastError() == cudaSuccess ? 0 : DSMC_ERR_CUDA;
}

}  // namespace dsmc
