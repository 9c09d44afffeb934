// chi-MLP surrogate (Sec. 3.4, Fig. nn_architecture; reading R9) on the
// tcgen05 tensor cores: inputs [ln(E_r)*, b/b_max] -> 512, 512, 512, 256, 128
// (SiLU) -> 1 (Softplus); the Softplus output y approximates ln(1 + chi),
// so chi = e^y - 1.  It synthesises the look-up table of Sec. 3.4.4.
//
// One persistent CTA of 17 warps per SM works on 128-row tiles.  The
// tile's activations stay in shared memory (bf16, K-major core matrices,
// 128 x 512 = 128 KB); the weights (1.36 MB, the same for every tile) stream
// from L2 in chunks of 16 K-columns x N rows, packed once in the MMA's
// operand layout (dsmc_chi_mlp_pack) so that each chunk is one contiguous
// bulk copy (cp.async.bulk, completion counted on an mbarrier), through a
// ring of five 16 KB buffers.  A producer warp issues the copies and the MMAs
// (M = 128, N = 256 per instruction, K = 16 per chunk, FP32 accumulators in
// all 512 TMEM columns) and recycles a buffer once the MMAs of the chunk
// two before the current one have completed (one lane issues; a warp of
// its own, so that no waiting lane of the same warp holds it back).  After a
// layer's last chunk the 16 epilogue warps read the accumulators back (warp w: TMEM lanes 32 (w % 4),
// a quarter of the columns), add the bias, apply SiLU and store the next
// layer's input as single bf16 terms; the fifth hidden layer's activations
// go straight into FP32 dot products with the output weights.
//
// Precision: the input enters as two bf16 terms (about 16 bits); hidden
// activations 1-4 are stored as single bf16 terms (a second term would not
// fit 128 rows x 512 columns twice in shared memory); accumulation in FP32.
#include <vector>

#include "internal.cuh"
#include "tc.cuh"

namespace dsmc {

namespace {

constexpr int kRows = 128;
constexpr int kEpiWarps = 16;                  // epilogue warps: 4 TMEM lane quadrants x 4 column groups
constexpr int kThr = (kEpiWarps + 1) * 32;     // + one producer warp (copies and MMAs)
constexpr int kNbuf = 5;
constexpr int kLag = 2;     // a buffer is recycled once the chunk kLag before the current one is done
constexpr int kChunkK = 16;
constexpr int kMmaLayers = 5;                       // hidden layers 1..5 on the tensor cores
// widths 2, 512, 512, 512, 256, 128, 1; K and N of the MMA layers (input padded to K = 16)
__host__ __device__ constexpr int dims_of(int i) {
  return i == 0 ? 2 : i <= 3 ? 512 : i == 4 ? 256 : i == 5 ? 128 : 1;
}
__host__ __device__ constexpr int k_of(int l) { return l == 0 ? 16 : l <= 3 ? 512 : 256; }
__host__ __device__ constexpr int n_of(int l) { return l <= 2 ? 512 : l == 3 ? 256 : 128; }
constexpr int kBiasTotal = 512 + 512 + 512 + 256 + 128 + 1;

__host__ __device__ constexpr int chunks_of(int l) { return k_of(l) / kChunkK; }
__host__ __device__ constexpr int chunk_bytes(int l) { return n_of(l) * kChunkK * 2; }
__host__ __device__ constexpr int chunks_per_tile() {
  return chunks_of(0) + chunks_of(1) + chunks_of(2) + chunks_of(3) + chunks_of(4);
}
// byte offset of layer l's first chunk in the packed weights
__host__ __device__ constexpr uint32_t layer_off(int l) {
  uint32_t o = 0;
  for (int q = 0; q < l; ++q) o += (uint32_t)(k_of(q) * n_of(q) * 2);
  return o;
}
constexpr uint32_t kWoutOff = layer_off(kMmaLayers);          // FP32 output weights [128]
constexpr uint32_t kPackedBytes = kWoutOff + 128 * 4;
constexpr int kPerTile = chunks_per_tile();                     // 113

// chunk index m of a CTA's sequence -> (layer, chunk within the layer)
__device__ __forceinline__ void chunk_id(int m, int* l, int* c) {
  int r = m % kPerTile, q = 0;
  while (r >= chunks_of(q)) { r -= chunks_of(q); ++q; }
  *l = q; *c = r;
}

// shared memory layout (bytes)
constexpr uint32_t kActOff = 0;                                  // 128 x 512 bf16
constexpr uint32_t kBufOff = kActOff + kRows * 512 * 2;          // kNbuf x 16 KB
constexpr uint32_t kBufBytes = 512 * kChunkK * 2;
constexpr uint32_t kBiasOff = kBufOff + kNbuf * kBufBytes;
constexpr uint32_t kWoOff = kBiasOff + ((kBiasTotal * 4 + 15) / 16) * 16;
constexpr uint32_t kYpOff = kWoOff + 128 * 4;                    // 4 column groups x 128 rows
constexpr uint32_t kBarOff = kYpOff + 4 * kRows * 4;             // full[kNbuf], empty[kNbuf], acc
constexpr uint32_t kTptrOff = kBarOff + (2 * kNbuf + 1) * 8;
constexpr uint32_t kFlagOff = kTptrOff + 8;
constexpr uint32_t kSmemBytes = kFlagOff + 16;

struct ChiArgs {
  const char* packed;
  const float* bias;
  int64_t n;
  const float* x;      // [n][2], or null (table mode)
  float* y;            // Softplus outputs, or null
  float* chi;          // e^y - 1, or null
  int32_t nb, nE;      // table mode: row g is node (g / nb, g % nb)
  int* status;
};

__device__ __forceinline__ float softplus_f(float z) { return fmaxf(z, 0.f) + log1pf(__expf(-fabsf(z))); }

}  // namespace

// ------------------------------------------------------------------ packing
// packed chunk (l, c): N_l rows x 16 K-columns in the K-major core-matrix
// layout (row n, column k at kmajor_offset(n, k, 16)); layer 1 (K = 2 in the
// network) holds W1[n][0], W1[n][1] in columns 0, 1 (the inputs' bf16 terms)
// and again in 2, 3 (their remainders); zeros elsewhere.
__global__ void k_chi_mlp_pack(const uint16_t* __restrict__ w, char* __restrict__ packed) {
  const int64_t total = (int64_t)layer_off(kMmaLayers) / 2;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total + 128;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (e >= total) {   // output weights W6[0][k] as FP32
      const int k = (int)(e - total);
      uint32_t src_off = 0;
      for (int q = 0; q < 5; ++q) src_off += (uint32_t)(dims_of(q) * dims_of(q + 1));
      ((float*)(packed + kWoutOff))[k] = __uint_as_float((uint32_t)w[src_off + k] << 16);
      continue;
    }
    int l = 0;
    int64_t r = e;
    while (r >= (int64_t)k_of(l) * n_of(l)) { r -= (int64_t)k_of(l) * n_of(l); ++l; }
    const int c = (int)(r / (n_of(l) * kChunkK));
    const int rem = (int)(r % (n_of(l) * kChunkK));
    // rem indexes the chunk's bytes / 2: invert kmajor_offset(n, k, 16)
    const int grp = rem / 128, in_grp = rem % 128;   // 8 rows x 16 columns per 256 bytes = 128 elements
    const int kc = (in_grp / 64), within = in_grp % 64;
    const int n = grp * 8 + within / 8, k = kc * 8 + within % 8;
    uint32_t src_off = 0;
    for (int q = 0; q < l; ++q) src_off += (uint32_t)(dims_of(q) * dims_of(q + 1));
    const int din = dims_of(l);
    uint16_t v = 0;
    if (l == 0) {
      if (k < 4) v = w[src_off + n * din + (k & 1)];
    } else {
      v = w[src_off + n * din + c * kChunkK + k];
    }
    ((uint16_t*)(packed + layer_off(l) + (uint32_t)c * chunk_bytes(l)))[tc::kmajor_offset(n, k, kChunkK) / 2] = v;
  }
}

// ------------------------------------------------------------------ forward
__global__ void __launch_bounds__(kThr, 1) k_chi_mlp(ChiArgs a) {
  extern __shared__ __align__(1024) char smem[];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int q = w & 3, cg = w >> 2;           // TMEM lane quadrant, column group
  const int row = q * 32 + lane;
  uint64_t* full = (uint64_t*)(smem + kBarOff);
  uint64_t* empty = full + kNbuf;
  uint64_t* acc_bar = full + 2 * kNbuf;
  volatile int* fail = (volatile int*)(smem + kFlagOff);
  const uint32_t sbase = tc::smem_u32(smem);
  float* bias = (float*)(smem + kBiasOff);
  float* wo = (float*)(smem + kWoOff);
  float* yp = (float*)(smem + kYpOff);
  for (int i = t; i < kBiasTotal; i += kThr) bias[i] = a.bias[i];
  for (int i = t; i < 128; i += kThr) wo[i] = ((const float*)(a.packed + kWoutOff))[i];
  if (w == 0) {
    tc::tmem_alloc((uint32_t*)(smem + kTptrOff), 512);
    tc::tmem_relinquish();
  }
  if (t == 0) {
    // full: the producer's expect-tx and the copy's bytes; empty: the commit
    // of the MMAs that read the buffer; acc: the commit of a layer's last MMAs
    for (int b = 0; b < kNbuf; ++b) { tc::mbar_init(full + b, 1); tc::mbar_init(empty + b, 1); }
    tc::mbar_init(acc_bar, 1);
    tc::mbar_fence_init();
    *fail = 0;
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *(volatile uint32_t*)(smem + kTptrOff);

  // Tiles blockIdx.x, blockIdx.x + gridDim.x, ...: every CTA streams the
  // whole weight sequence once per tile into its own buffers.
  const int64_t n_tiles = (a.n + kRows - 1) / kRows;
  const int my_its = (int64_t)blockIdx.x < n_tiles ? (int)((n_tiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;
  const int total = my_its * kPerTile;     // chunks this CTA consumes
  int issued = 0, consumed = 0;            // producer warp's counters
  // producer lane 0: chunk m into buffer m % kNbuf
  auto issue_copy = [&](int m) {
    int l, c;
    chunk_id(m, &l, &c);
    const int b = m % kNbuf;
    tc::mbar_arrive_expect_tx(full + b, (uint32_t)chunk_bytes(l));
    tc::bulk_g2s(sbase + kBufOff + (uint32_t)b * kBufBytes, a.packed + layer_off(l) + (uint32_t)c * chunk_bytes(l),
                 (uint32_t)chunk_bytes(l), full + b);
  };
  if (w == kEpiWarps) {
    if (lane == 0)
      for (int m = 0; m < kNbuf && m < total; ++m) issue_copy(m);
    issued = kNbuf < total ? kNbuf : total;
  }

  uint32_t acc_phase = 0;
  bool ok = true;
  for (int it = 0; it < my_its && ok; ++it) {
    const int64_t tile = (int64_t)blockIdx.x + (int64_t)it * gridDim.x;
    // input row (threads 0..127): [x0 hi, x1 hi, x0 lo, x1 lo, 0 ...] as a K = 16 tile
    if (t < kRows) {
      const int64_t gr = tile * kRows + t;
      float x0 = 0.f, x1 = 0.f;
      if (gr < a.n) {
        if (a.x) { x0 = a.x[2 * gr]; x1 = a.x[2 * gr + 1]; }
        else {
          x0 = (float)(gr / a.nb) / (float)(a.nE - 1);
          x1 = (float)(gr % a.nb) / (float)(a.nb - 1);
        }
      }
      const uint32_t hi = tc::pack_bf16x2(x0, x1);
      const float h0 = __uint_as_float(hi << 16), h1 = __uint_as_float(hi & 0xFFFF0000u);
      const uint32_t lo = tc::pack_bf16x2(x0 - h0, x1 - h1);
      tc::st_shared_v4(sbase + kActOff + tc::kmajor_offset(t, 0, kChunkK), hi, lo, 0u, 0u);
      tc::st_shared_v4(sbase + kActOff + tc::kmajor_offset(t, 8, kChunkK), 0u, 0u, 0u, 0u);
    }
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    float2 yq = make_float2(0.f, 0.f);
    uint32_t boff = 0;
    for (int l = 0; l < kMmaLayers; ++l) {
      if (w == kEpiWarps) {   // producer warp: all lanes follow the loop, lane 0 issues
        tc::fence_after();
        const uint32_t sbo_a = (uint32_t)k_of(l) * 16;
        const int nh = n_of(l) > 256 ? 2 : 1, nn = n_of(l) > 256 ? 256 : n_of(l);
        const uint32_t idesc = tc::idesc_bf16(kRows, nn);
        for (int c = 0; c < chunks_of(l) && ok; ++c) {
          const int m = consumed;
          const int b = m % kNbuf;
          // the warp agrees on every wait's outcome
          if (!__all_sync(0xffffffffu, tc::mbar_wait(full + b, (uint32_t)(m / kNbuf) & 1u, a.status, kBarrierLimitNs))) {
            ok = false;
            break;
          }
          if (lane == 0) {
            const uint32_t bb = sbase + kBufOff + (uint32_t)b * kBufBytes;
            for (int h = 0; h < nh; ++h)
              tc::mma_bf16(tmem + (uint32_t)(256 * h), tc::sdesc(sbase + kActOff + 256u * (uint32_t)c, 128, sbo_a),
                           tc::sdesc(bb + (uint32_t)h * 8192u, 128, 256), idesc, c > 0);
            tc::commit(empty + b);
          }
          __syncwarp();
          ++consumed;
          // recycle the buffer of the chunk kLag before this one (its MMAs
          // finish ahead of the ones issued since, which keep the tensor pipe
          // busy meanwhile)
          if (m >= kLag && issued < total) {
            const int mp = m - kLag;
            if (!__all_sync(0xffffffffu,
                            tc::mbar_wait(empty + mp % kNbuf, (uint32_t)(mp / kNbuf) & 1u, a.status, kBarrierLimitNs))) {
              ok = false;
              break;
            }
            if (lane == 0) issue_copy(issued);
            __syncwarp();
            ++issued;
          }
        }
        if (lane == 0) {
          if (ok) tc::commit(acc_bar);
          else *fail = 1;
        }
        __syncwarp();
      }
      // every thread waits for the layer's accumulators; the block agrees
      const bool got = w == kEpiWarps || tc::mbar_wait(acc_bar, acc_phase, a.status, kBarrierLimitNs);
      acc_phase ^= 1u;
      if (!__syncthreads_and(got && !*fail)) { ok = false; break; }
      tc::fence_after();
      if (w < kEpiWarps) {
        const int ncols = n_of(l) / 4, cbeg = cg * ncols, npieces = ncols / 16;
        const uint32_t lane_tm = tmem + ((uint32_t)(q * 32) << 16);
        const float* bl = bias + boff;
        const bool last = l == kMmaLayers - 1;
        const uint32_t knext = (uint32_t)n_of(l);
        uint32_t ra[16], rb[16];
        tc::ld16_async(lane_tm + (uint32_t)cbeg, ra);
        tc::wait_ld16(ra);
#pragma unroll 1
        for (int pc = 0; pc < npieces; pc += 2) {
#pragma unroll
          for (int half = 0; half < 2; ++half) {
            uint32_t* cur = half ? rb : ra;
            uint32_t* nxt = half ? ra : rb;
            const int c0 = cbeg + 16 * (pc + half);
            const bool more = pc + half + 1 < npieces;
            if (more) tc::ld16_async(lane_tm + (uint32_t)(c0 + 16), nxt);
            float2 v[8];
            const float2* b2 = (const float2*)(bl + c0);
#pragma unroll
            for (int k = 0; k < 8; ++k)
              v[k] = __fadd2_rn(make_float2(__uint_as_float(cur[2 * k]), __uint_as_float(cur[2 * k + 1])), b2[k]);
#pragma unroll
            for (int k = 0; k < 8; k += 2) tc::silu4x2(v[k], v[k + 1]);
            if (last) {
              const float2* w2 = (const float2*)(wo + c0);
#pragma unroll
              for (int k = 0; k < 8; ++k) yq = __ffma2_rn(v[k], w2[k], yq);
            } else {
              uint32_t pk[8];
#pragma unroll
              for (int k = 0; k < 8; ++k) pk[k] = tc::pack_bf16x2(v[k].x, v[k].y);
              tc::st_shared_v4(sbase + kActOff + tc::kmajor_offset(row, c0, (int)knext), pk[0], pk[1], pk[2], pk[3]);
              tc::st_shared_v4(sbase + kActOff + tc::kmajor_offset(row, c0 + 8, (int)knext), pk[4], pk[5], pk[6], pk[7]);
            }
            if (more) tc::wait_ld16(nxt);
          }
        }
      }
      boff += (uint32_t)n_of(l);
      tc::fence_async_smem();
      tc::fence_before();
      __syncthreads();
    }
    if (!ok) break;
    // output layer: the four column groups' partial dot products, bias, Softplus
    if (w < kEpiWarps) yp[cg * kRows + row] = yq.x + yq.y;
    __syncthreads();
    if (t < kRows) {
      const int64_t gr = tile * kRows + t;
      if (gr < a.n) {
        const float z = yp[t] + yp[kRows + t] + yp[2 * kRows + t] + yp[3 * kRows + t] + bias[boff];
        const float y = softplus_f(z);
        if (a.y) a.y[gr] = y;
        if (a.chi) a.chi[gr] = expm1f(y);
      }
    }
    __syncthreads();
  }
  // on failure: let the copies this CTA's buffers expect land (bounded)
  // before its shared memory and TMEM are released
  if (w == kEpiWarps && lane == 0 && !ok) {
    for (int m = consumed; m < issued; ++m)
      tc::mbar_wait(full + m % kNbuf, (uint32_t)(m / kNbuf) & 1u, a.status, kBarrierLimitNs);
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (w == 0) tc::tmem_dealloc(tmem, 512);
}

// ------------------------------------------------------------------ host side
size_t chi_mlp_packed_size() { return kPackedBytes; }

int launch_chi_mlp_pack(Ctx* c, const uint16_t* w_bits, void* packed, cudaStream_t s) {
  k_chi_mlp_pack<<<sm_count(c) * 4, 256, 0, s>>>(w_bits, (char*)packed);
  count_launches(c, 1);
  return cudaGetLastError() == cudaSuccess ? 0 : DSMC_ERR_CUDA;
}

static int launch_chi_mlp(Ctx* c, const ChiArgs& a, cudaStream_t s) {
  if (a.n == 0) return 0;
  if (cudaFuncSetAttribute((const void*)k_chi_mlp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes) !=
      cudaSuccess)
    return record(c, DSMC_ERR_CUDA, "chi_mlp: shared memory attribute");
  // one wave of persistent CTAs, one per SM (223 KB of shared memory each)
  const int64_t tiles = (a.n + kRows - 1) / kRows;
  const int64_t grid = tiles < sm_count(c) ? tiles : sm_count(c);
  k_chi_mlp<<<(unsigned)grid, kThr, kSmemBytes, s>>>(a);
  count_launches(c, 1);
  return cudaGetLastError() == cudaSuccess ? 0 : DSMC_ERR_CUDA;
}

int launch_chi_mlp_forward(Ctx* c, const void* packed, const float* bias, int64_t n, const float* x, float* y,
                           float* chi, cudaStream_t s) {
  ChiArgs a = {};
  a.packed = (const char*)packed; a.bias = bias; a.n = n; a.x = x; a.y = y; a.chi = chi;
  a.status = status_ptr(c);
  return launch_chi_mlp(c, a, s);
}

int launch_chi_mlp_table(Ctx* c, const void* packed, const float* bias, int32_t nb, int32_t nE, float* table,
                         cudaStream_t s) {
  ChiArgs a = {};
  a.packed = (const char*)packed; a.bias = bias; a.n = (int64_t)nb * nE; a.chi = table;
  a.nb = nb; a.nE = nE;
  a.status = status_ptr(c);
  return launch_chi_mlp(c, a, s);
}

}  // namespace dsmc
