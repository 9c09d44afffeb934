// No-Time-Counter pair selection (Sec. 2.2) and the conflict-free round
// schedule of the accepted pairs.
//
//   k_sel_count   warp per cell: M = floor(1/2 N(N-1) F_N/V_c (sg)max dt + U),
//                 evaluate every candidate, count acceptances, new (sg)max
//   scan          counts -> per-cell pair offsets
//   k_sel_emit    warp per cell: the accepted candidates (from the count
//                 pass's accept bits) compacted in candidate order and their
//                 particles drawn, then rounds in candidate order:
//                 round = 1 + max(last[i], last[j])
//   scan          per-round counts -> round offsets
//   k_sel_rcount, k_sel_rscan, k_sel_scatter: stable round-major regrouping
//                 of the pairs (cell-major candidate order inside a round),
//                 each with the rounds of the previous pairs of its particles
//
// The accept decision and M are taken in FP64 with explicitly rounded
// operations (no contraction into FMA), in the operation order of the
// definition, so that they agree exactly with any other correctly rounded
// evaluation of the same formula.
#include "select.cuh"

namespace dsmc {

constexpr int kSelWarps = 8;

// Words of accept bits per cell: ceil(M/32) for the cell's candidate count M.
__global__ void k_sel_nwords(SelArgs a) {
  if (a.step_dev) a.step = *a.step_dev;
  unsigned long long total = 0;
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < a.n_cells; k += gridDim.x * blockDim.x) {
    const int32_t N = a.cs[k + 1] - a.cs[k];
    int bad = 0;
    const int32_t M = N < 2 ? 0 : ntc_count(a, k, N, &bad);
    if (bad) set_status(a.status, DSMC_ERR_CAPACITY);
    a.ncand[k] = M;
    total += (unsigned long long)M;
    const int64_t words = ((int64_t)M + 31) / 32;
    a.wcnt[k] = (int32_t)(words <= a.words_cap ? words : 0);  // too many: never kept
  }
  // one atomic per warp for the step's candidate count
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
  if ((threadIdx.x & 31) == 0 && total) atomicAdd(a.n_cand, total);
}

// Stage the cell's velocities (FP32) in this warp's shared-memory slice
// (none when sm is null: the candidates then read FP64 from global memory)
// and derive the screening constants.
__device__ __forceinline__ CellView stage_cell(const SelArgs& a, float4* sm, int32_t base, int32_t N,
                                               double sgk, int lane) {
  CellView cv;
  cv.x = cv.y = cv.z = nullptr;
  cv.v4 = nullptr;
  float vmax = 0.f;
  if (sm && N <= kStage) {
    for (int32_t t = lane; t < N; t += 32) {
      const float fx = f64_to_f32(a.vx[base + t]), fy = f64_to_f32(a.vy[base + t]), fz = f64_to_f32(a.vz[base + t]);
      sm[t] = make_float4(fx, fy, fz, 0.f);
      vmax = fmaxf(vmax, fmaxf(fabsf(fx), fmaxf(fabsf(fy), fabsf(fz))));
    }
    cv.v4 = sm;
  } else {
    for (int32_t t = lane; t < N; t += 32)
      vmax = fmaxf(vmax, (float)fmax(fabs(a.vx[base + t]), fmax(fabs(a.vy[base + t]), fabs(a.vz[base + t]))));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
  __syncwarp();
  // each velocity carries <= |v| 2^-24 rounding; g over three differences
  cv.dg = 4.0f * vmax * 5.9604645e-8f;
  cv.sgmax32 = f64_to_f32(sgk);
  cv.inv_sgmax32 = 1.f / cv.sgmax32;
  cv.thr_raise = cv.sgmax32 * (1.f - 3e-4f);
  return cv;
}

// One cell by the whole warp (candidates 32 at a time).
__device__ __forceinline__ void count_cell(const SelArgs& a, float4* stage, int32_t k, int lane) {
  const int32_t base = a.cs[k], N = a.cs[k + 1] - base;
  const double sgk = a.sgmax[k];
  if (N < 2) {
    if (lane == 0) { a.counts[k] = 0; a.sgnew[k] = sgk; }
    return;
  }
  const int32_t M = a.ncand[k];   // from k_sel_nwords (which reports an overflow)
  const CellView cv = stage_cell(a, stage, base, N, sgk, lane);
  int acc = 0;
  // The maximum is taken on the bit patterns: for non-negative doubles the
  // int64 order is the numeric order, and it keeps the FP64 pipe free
  // (candidates that cannot raise the maximum carry -1.0, a negative int64).
  long long best = __double_as_longlong(sgk);
  const int64_t w0 = a.wofs[k];
  const bool keep = bits_kept(a, k, M);
  for (int32_t c0 = 0; c0 < M; c0 += 32) {
    const int32_t m = c0 + lane;
    int32_t i, j;
    double sg = -1.0;
    const bool ok = m < M && candidate(a, cv, CellRef{a.vx, a.vy, a.vz, base}, k, N, m, sgk, &i, &j, &sg);
    acc += ok;
    best = max(best, __double_as_longlong(sg));
    const unsigned mask = __ballot_sync(0xffffffffu, ok);
    if (keep && lane == 0) a.bits[w0 + c0 / 32] = mask;
  }
  acc = warp_sum_i(acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
  if (lane == 0) {
    a.counts[k] = acc;
    a.sgnew[k] = __longlong_as_double(best);
  }
  __syncwarp();
}

// Two cells of at most 16 candidates each, one per half-warp (lanes 16h ..
// 16h + 15): most cells of a dilute gas draw so few candidates that a whole
// warp per cell would leave half its lanes idle and pay the per-cell work
// twice.  Called by the whole warp; kk[h] = the half's cell (n_cells: none).
__device__ __forceinline__ void count_pair(const SelArgs& a, float4* stage, const int32_t kk[2], int lane) {
  const int h = lane >> 4, hl = lane & 15;
  const int32_t k = kk[h];
  const bool valid = k < a.n_cells;
  const int32_t base = valid ? a.cs[k] : 0, N = valid ? a.cs[k + 1] - base : 0;
  const double sgk = valid ? a.sgmax[k] : 0.0;
  const int32_t M = N >= 2 ? a.ncand[k] : 0;
  // the half's FP32 copy and screening constants (as stage_cell, 16 lanes)
  float4* sm = stage + h * (kStage / 2);
  float vmax = 0.f;
  for (int32_t t = hl; t < N; t += 16) {
    const float fx = f64_to_f32(a.vx[base + t]), fy = f64_to_f32(a.vy[base + t]), fz = f64_to_f32(a.vz[base + t]);
    sm[t] = make_float4(fx, fy, fz, 0.f);
    vmax = fmaxf(vmax, fmaxf(fabsf(fx), fmaxf(fabsf(fy), fabsf(fz))));
  }
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
  __syncwarp();
  CellView cv;
  cv.x = cv.y = cv.z = nullptr;
  cv.v4 = sm;
  cv.dg = 4.0f * vmax * 5.9604645e-8f;
  cv.sgmax32 = f64_to_f32(sgk);
  cv.inv_sgmax32 = 1.f / cv.sgmax32;
  cv.thr_raise = cv.sgmax32 * (1.f - 3e-4f);
  int32_t i, j;
  double sg = -1.0;
  const bool ok = hl < M && candidate(a, cv, CellRef{a.vx, a.vy, a.vz, base}, k, N, hl, sgk, &i, &j, &sg);
  const unsigned mask = __ballot_sync(0xffffffffu, ok);
  const unsigned word = h ? mask >> 16 : mask & 0xFFFFu;
  long long best = valid ? __double_as_longlong(sgk) : 0ll;
  best = max(best, __double_as_longlong(sg));
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
  if (hl == 0 && valid) {
    a.counts[k] = N >= 2 ? __popc(word) : 0;
    a.sgnew[k] = __longlong_as_double(best);
    if (N >= 2 && M > 0 && bits_kept(a, k, M)) a.bits[a.wofs[k]] = word;
  }
  __syncwarp();
}

// Warp per pair of consecutive cells: both by half-warps when each draws at
// most 16 candidates (and fits half the staging slice), else one after the
// other by the whole warp.
__global__ void __launch_bounds__(kSelWarps * 32, 4) k_sel_count(SelArgs a) {
  if (a.step_dev) a.step = *a.step_dev;
  __shared__ float4 stage[kSelWarps][kStage];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int32_t warps = gridDim.x * kSelWarps;
  const int32_t npairs = (a.n_cells + 1) / 2;
  for (int32_t kp = blockIdx.x * kSelWarps + wid; kp < npairs; kp += warps) {
    const int32_t kk[2] = {2 * kp, 2 * kp + 1 < a.n_cells ? 2 * kp + 1 : a.n_cells};
    bool small = true;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (kk[h] >= a.n_cells) continue;
      const int32_t N = a.cs[kk[h] + 1] - a.cs[kk[h]];
      if (N >= 2 && (N > kStage / 2 || a.ncand[kk[h]] > 16)) small = false;
    }
    if (small) {
      count_pair(a, stage[wid], kk, lane);
    } else {
      count_cell(a, stage[wid], kk[0], lane);
      if (kk[1] < a.n_cells) count_cell(a, stage[wid], kk[1], lane);
    }
  }
}

constexpr int kEmitWarps = 8;
constexpr int kEmitWords = 16;    // accept-bit words expanded per step (512 candidates)

// Warp per cell.  The accepted candidates come from the count pass's accept
// bits (kEmitWords words at a time, compacted in candidate order into the
// warp's list); their particles are drawn 32 at a time (the generator runs
// once per accepted candidate with every lane busy) and each batch of 32
// pairs gets its rounds at once (batch_rounds), so no per-cell pair buffer
// is kept.  A cell whose bits were not kept re-evaluates its candidates
// from the FP64 velocities; a cell of more than kStage particles takes its
// rounds on one lane from global memory.
__global__ void __launch_bounds__(kEmitWarps * 32, 4) k_sel_emit(SelArgs a) {
  if (a.step_dev) a.step = *a.step_dev;
  __shared__ uint32_t slist[kEmitWarps][kEmitWords * 32];  // accepted candidate indices
  __shared__ uint32_t smsk[kEmitWarps][kStage];            // per-particle lane masks (batch_rounds)
  __shared__ uint16_t slast[kEmitWarps][kStage];           // last round of each particle (+1; 0 = none)
  __shared__ int hist[DSMC_MAX_ROUNDS];
  __shared__ int rmax_blk;
  for (int t = threadIdx.x; t < DSMC_MAX_ROUNDS; t += blockDim.x) hist[t] = 0;
  if (threadIdx.x == 0) rmax_blk = 0;
  __syncthreads();
  const int64_t total = a.offs[a.n_cells];
  const bool over = total > a.capacity;
  if (over && blockIdx.x == 0 && threadIdx.x == 0) set_status(a.status, DSMC_ERR_CAPACITY);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  uint32_t* list = slist[wid];
  uint32_t* msk = smsk[wid];
  uint16_t* last = slast[wid];
  const int32_t warps = gridDim.x * kEmitWarps;
  int rm = -1;
  // one cell by the whole warp
  auto emit_cell = [&](const int32_t k) {
    const int32_t base = a.cs[k], N = a.cs[k + 1] - base;
    if (N < 2) return;
    const double sgk = a.sgmax[k];
    const int32_t M = a.ncand[k];
    const bool from_bits = bits_kept(a, k, M);
    const int64_t w0 = a.wofs[k];
    const int32_t p0 = a.offs[k], p1 = a.offs[k + 1];
    const bool local = N <= kStage;
    if (local) {
      for (int32_t t = lane; t < N; t += 32) { last[t] = 0; msk[t] = 0u; }
    } else {
      for (int32_t t = lane; t < N; t += 32) a.last[base + t] = -1;
    }
    __syncwarp();
    int32_t pos = p0;
    int cm = -1;   // this lane's largest round of the cell
    // one batch of up to 32 accepted pairs in candidate order: lane t holds
    // pair pos + t (act), candidate m, particles i, j
    auto batch = [&](bool act, int32_t m, int32_t i, int32_t j, int cnt) {
      const int32_t q = pos + lane;
      if (act) a.tmp[q] = make_int4(base + i, base + j, k, m);
      if (local) {
        int Li, Lj;
        const int r = batch_rounds(act, (uint32_t)i, (uint32_t)j, msk, last, a.status, &Li, &Lj);
        if (act) {
          a.tmp_round[q] = r;
          a.tmp_dep[q] = (uint32_t)Li | ((uint32_t)Lj << 16);
          rm = r > rm ? r : rm;
          cm = r > cm ? r : cm;
        }
        if (act) atomicAdd(&hist[r], 1);
        __syncwarp();
      }
      pos += cnt;
    };
    if (from_bits) {
      const int32_t nwords = (M + 31) / 32;
      for (int32_t wb = 0; wb < nwords; wb += kEmitWords) {
        const int nq = min(kEmitWords, nwords - wb);
        const uint32_t bw = lane < nq ? a.bits[w0 + wb + lane] : 0u;
        const int cnt = __popc(bw);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < kEmitWords; o <<= 1) {
          const int v = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += v;
        }
        const int tot = __shfl_sync(0xffffffffu, incl, kEmitWords - 1);
        const int before = incl - cnt;
        for (int q = 0; q < nq; ++q) {
          const uint32_t wq = __shfl_sync(0xffffffffu, bw, q);
          const int bq = __shfl_sync(0xffffffffu, before, q);
          if ((wq >> lane) & 1u) list[bq + __popc(wq & lt)] = (uint32_t)((wb + q) * 32 + lane);
        }
        __syncwarp();
        for (int t0 = 0; t0 < tot; t0 += 32) {
          const int t = t0 + lane;
          const bool act = t < tot;
          int32_t m = 0, i = 0, j = 1;
          if (act) {
            m = (int32_t)list[t];
            cand_ij(a, k, N, m, &i, &j);
          }
          batch(act, m, i, j, min(32, tot - t0));
        }
        __syncwarp();
      }
    } else {
      // bits not kept: re-evaluate every candidate (FP64 velocities from global memory)
      CellView cv = stage_cell(a, nullptr, base, N, sgk, lane);
      for (int32_t c0 = 0; c0 < M; c0 += 32) {
        const int32_t m = c0 + lane;
        int32_t i = 0, j = 1;
        double sg;
        const bool ok = m < M && candidate(a, cv, CellRef{a.vx, a.vy, a.vz, base}, k, N, m, sgk, &i, &j, &sg);
        const unsigned mask = __ballot_sync(0xffffffffu, ok);
        // compact the accepted lanes into lanes 0.. in candidate order
        int32_t cm = 0, ci = 0, cj = 1;
        for (int q = 0; q < 32; ++q) {
          if (!((mask >> q) & 1u)) continue;
          const int r = __popc(mask & ((1u << q) - 1u));
          const int32_t vm = __shfl_sync(0xffffffffu, m, q), vi = __shfl_sync(0xffffffffu, i, q),
                        vj = __shfl_sync(0xffffffffu, j, q);
          if (lane == r) { cm = vm; ci = vi; cj = vj; }
        }
        const int cnt = __popc(mask);
        batch(lane < cnt, cm, ci, cj, cnt);
      }
    }
    __syncwarp();   // the cell's pairs (written by all lanes) before lane 0 reads them
    if (!local && lane == 0) {
      for (int32_t p = p0; p < p1; ++p) {
        const int4 q = a.tmp[p];
        const int li = a.last[q.x], lj = a.last[q.y];
        int r = 1 + (li > lj ? li : lj);
        if (r >= DSMC_MAX_ROUNDS) { set_status(a.status, DSMC_ERR_UNSUPPORTED); r = DSMC_MAX_ROUNDS - 1; }
        a.last[q.x] = r;
        a.last[q.y] = r;
        a.tmp_round[p] = r;
        a.tmp_dep[p] = (uint32_t)(li + 1) | ((uint32_t)(lj + 1) << 16);
        atomicAdd(&hist[r], 1);
        rm = r > rm ? r : rm;
        cm = r > cm ? r : cm;
      }
    }
    if (a.order) {
      // the cell's last round beside each of its pairs' rounds
      __syncwarp();
      const int last_round = __reduce_max_sync(0xffffffffu, cm);
      for (int32_t p = p0 + lane; p < p1; p += 32) a.tmp_round[p] |= last_round << 16;
    }
    if (lane == 0) a.sgmax[k] = a.sgnew[k];
    __syncwarp();
  };
  // two cells of at most 16 candidates each (their accept bits kept, at most
  // kStage/2 particles), one per half-warp: the accepted candidates of a
  // cell fit one batch of its 16 lanes, and the lane masks of the round
  // assignment stay within a half since each half has its own particles
  auto emit_pair = [&](const int32_t kk[2]) {
    const int h = lane >> 4, hl = lane & 15;
    const int32_t k = kk[h];
    const bool valid = k < a.n_cells;
    const int32_t base = valid ? a.cs[k] : 0, N = valid ? a.cs[k + 1] - base : 0;
    uint32_t* mh = msk + h * (kStage / 2);
    uint16_t* lh = last + h * (kStage / 2);
    for (int32_t t = hl; t < N; t += 16) { lh[t] = 0; mh[t] = 0u; }
    __syncwarp();
    const bool live = N >= 2;
    const int32_t M = live ? a.ncand[k] : 0;
    const uint32_t word = M > 0 ? a.bits[a.wofs[k]] : 0u;
    const bool act = hl < __popc(word);
    int32_t m = 0, i = 0, j = 1;
    if (act) {
      uint32_t w = word;   // the hl-th accepted candidate, in candidate order
      for (int c = 0; c < hl; ++c) w &= w - 1u;
      m = __ffs(w) - 1;
      cand_ij(a, k, N, m, &i, &j);
    }
    const int32_t q = (live ? a.offs[k] : 0) + hl;
    if (act) a.tmp[q] = make_int4(base + i, base + j, k, m);
    int Li, Lj;
    const int r = batch_rounds(act, (uint32_t)i, (uint32_t)j, mh, lh, a.status, &Li, &Lj);
    int cm = act ? r : -1;   // the half's cell's last round (shuffles within the half)
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) cm = max(cm, __shfl_xor_sync(0xffffffffu, cm, o));
    if (act) {
      a.tmp_round[q] = a.order ? (r | (cm << 16)) : r;
      a.tmp_dep[q] = (uint32_t)Li | ((uint32_t)Lj << 16);
      rm = r > rm ? r : rm;
      atomicAdd(&hist[r], 1);
    }
    __syncwarp();
    if (hl == 0 && live) a.sgmax[k] = a.sgnew[k];
    __syncwarp();
  };
  const int32_t npairs = (a.n_cells + 1) / 2;
  for (int32_t kp = blockIdx.x * kEmitWarps + wid; kp < npairs && !over; kp += warps) {
    const int32_t kk[2] = {2 * kp, 2 * kp + 1 < a.n_cells ? 2 * kp + 1 : a.n_cells};
    bool small = true;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (kk[h] >= a.n_cells) continue;
      const int32_t N = a.cs[kk[h] + 1] - a.cs[kk[h]];
      if (N < 2) continue;
      const int32_t M = a.ncand[kk[h]];
      if (N > kStage / 2 || M > 16 || !bits_kept(a, kk[h], M)) small = false;
    }
    if (small) {
      emit_pair(kk);
    } else {
      emit_cell(kk[0]);
      if (kk[1] < a.n_cells) emit_cell(kk[1]);
    }
  }
  rm = __reduce_max_sync(0xffffffffu, rm);
  if (lane == 0 && rm >= 0) atomicMax(&rmax_blk, rm + 1);
  __syncthreads();
  // per-round counts (the level counts, which need the step's round count,
  // come from k_sel_rcount)
  if (!a.order)
    for (int t = threadIdx.x; t < DSMC_MAX_ROUNDS; t += blockDim.x)
      if (hist[t]) atomicAdd(a.round_count + t, hist[t]);
  if (threadIdx.x == 0 && rmax_blk > 0) atomicMax(a.n_rounds, rmax_blk);
}

constexpr int kScatterChunk = 4096;

// Stable round-major regrouping of the cell-major pair list, in three
// kernels over chunks of kScatterChunk pairs: per chunk and round counts
// (cnt[r][chunk]), their exclusive scan along the chunks of each round plus
// the round's offset, then each chunk writes its pairs in order.  Inside a
// round the pairs keep the cell-major candidate order, so the list is
// deterministic and the pairs of a round's first cells come first.
//
// On a capacity overflow the emit pass skipped every cell; k_sel_rcount
// then commits the new (sigma g)_max of every cell instead (cells with
// fewer than two particles keep theirs).
__global__ void __launch_bounds__(256)
k_sel_rcount(const int32_t* __restrict__ tmp_round, const int32_t* __restrict__ offs, int32_t n_cells,
             int64_t capacity, const int32_t* __restrict__ n_rounds, int32_t n_chunks, int32_t* __restrict__ cnt,
             const double* __restrict__ sgnew, double* __restrict__ sgmax, int order,
             int32_t* __restrict__ level_count) {
  __shared__ int hist[DSMC_MAX_ROUNDS];
  const int64_t total = offs[n_cells];
  if (total > capacity) {
    for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n_cells; k += gridDim.x * blockDim.x)
      sgmax[k] = sgnew[k];
    return;
  }
  const int64_t p0 = (int64_t)blockIdx.x * kScatterChunk;
  if (p0 >= total) return;
  const int64_t p1 = p0 + kScatterChunk < total ? p0 + kScatterChunk : total;
  const int R = *n_rounds;
  for (int t = threadIdx.x; t < R; t += blockDim.x) hist[t] = 0;
  __syncthreads();
  for (int64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
    const int t = tmp_round[p];
    atomicAdd(&hist[order ? (t & 0xFFFF) + R - 1 - (t >> 16) : t], 1);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < R; t += blockDim.x) {
    cnt[(size_t)t * n_chunks + blockIdx.x] = hist[t];
    if (order && hist[t]) atomicAdd(level_count + t, hist[t]);
  }
}

// Block r: exclusive scan of cnt[r][0..chunks) + the offset of round r (in
// place).  The round offsets (exclusive scan of the per-round counts) are
// formed here too: block r sums the counts of rounds < r, and block 0
// writes the whole list.
__device__ __forceinline__ int block_sum_256(int v, int* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  int t = 0;
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
  return t;
}

__global__ void __launch_bounds__(256)
k_sel_rscan(const int32_t* __restrict__ offs, int32_t n_cells, int64_t capacity,
            const int32_t* __restrict__ n_rounds, const int32_t* __restrict__ round_count,
            int32_t* __restrict__ round_off, int32_t n_chunks, int32_t* __restrict__ cnt) {
  __shared__ int warp_tot[8];
  __shared__ int red[8];
  __shared__ int carry;
  const int64_t total = offs[n_cells];
  if (total > capacity || (int)blockIdx.x >= *n_rounds) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (blockIdx.x == 0) {
    // round_off[0..DSMC_MAX_ROUNDS]: kPer consecutive counts per thread
    constexpr int kPer = (DSMC_MAX_ROUNDS + 255) / 256;
    int v[kPer], sum = 0;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int r = threadIdx.x * kPer + q;
      v[q] = r < DSMC_MAX_ROUNDS ? round_count[r] : 0;
      sum += v[q];
    }
    int x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    int run = x - sum;
    for (int q = 0; q < w; ++q) run += warp_tot[q];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int r = threadIdx.x * kPer + q;
      if (r < DSMC_MAX_ROUNDS) round_off[r] = run;
      run += v[q];
    }
    if (threadIdx.x == blockDim.x - 1) round_off[DSMC_MAX_ROUNDS] = run;   // the total
    __syncthreads();
  }
  int part = 0;
  for (int q = threadIdx.x; q < (int)blockIdx.x; q += blockDim.x) part += round_count[q];
  part = block_sum_256(part, red);
  const int chunks = (int)((total + kScatterChunk - 1) / kScatterChunk);
  int32_t* row = cnt + (size_t)blockIdx.x * n_chunks;
  if (threadIdx.x == 0) carry = part;
  __syncthreads();
  for (int c0 = 0; c0 < chunks; c0 += blockDim.x) {
    const int c = c0 + threadIdx.x;
    const int v = c < chunks ? row[c] : 0;
    int x = v;  // inclusive scan in the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    int before = carry;
    for (int q = 0; q < w; ++q) before += warp_tot[q];
    if (c < chunks) row[c] = before + x - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = before + x;
    __syncthreads();
  }
}

// Block (16 warps) per chunk; warp w owns the chunk's w-th sixteenth, its
// rounds loaded first.  Stable ranks without a shared-memory round trip per
// batch: in each batch of 32 pairs the lanes of equal round find each other
// from ballots over the round's bits, the lowest adds the group's size to the warp's
// counter of that round (atomic, ordered across batches by __syncwarp) and
// keeps the old value; once the counts are complete they become per-warp
// starting positions (warps in order after the chunk's base), and each
// pair goes to start + its leader's old value + its rank in the group.
// The counters live in dynamic shared memory, kScatterWarps x n_rounds.
constexpr int kScatterWarps = 16;
constexpr int kScatterPer = kScatterChunk / kScatterWarps / 32;

__global__ void __launch_bounds__(kScatterWarps * 32, 2)
k_sel_scatter(const int4* __restrict__ tmp, const int32_t* __restrict__ tmp_round,
              const uint32_t* __restrict__ tmp_dep, const int32_t* __restrict__ offs, int32_t n_cells,
              int64_t capacity, const int32_t* __restrict__ n_rounds, int32_t n_chunks,
              const int32_t* __restrict__ base, int4* __restrict__ out, uint32_t* __restrict__ deps, int order) {
  extern __shared__ int swh[];   // [kScatterWarps][R]
  const int64_t total = offs[n_cells];
  if (total > capacity) return;
  const int64_t p0 = (int64_t)blockIdx.x * kScatterChunk;
  if (p0 >= total) return;
  const int64_t p1 = p0 + kScatterChunk < total ? p0 + kScatterChunk : total;
  const int R = *n_rounds;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  for (int t = threadIdx.x; t < kScatterWarps * R; t += blockDim.x) swh[t] = 0;
  const int64_t s0 = p0 + (int64_t)w * (kScatterPer * 32);
  int rr[kScatterPer];
#pragma unroll
  for (int j = 0; j < kScatterPer; ++j) {
    const int64_t p = s0 + j * 32 + lane;
    const int t = p < p1 ? tmp_round[p] : -1;
    rr[j] = order && t >= 0 ? (t & 0xFFFF) + R - 1 - (t >> 16) : t;
  }
  __syncthreads();
  int old[kScatterPer];
  uint32_t pk[kScatterPer];   // leader lane | rank in the group << 5
#pragma unroll
  for (int j = 0; j < kScatterPer; ++j) {
    // lanes of equal round (or without a pair): one ballot per bit of the
    // round numbers in use (the match instruction measured slower)
    unsigned peers = __ballot_sync(0xffffffffu, rr[j] >= 0);
    if (rr[j] < 0) peers = ~peers;
    for (int bit = 0; (1 << bit) < R; ++bit) {
      const unsigned m = __ballot_sync(0xffffffffu, (rr[j] >> bit) & 1);
      peers &= ((rr[j] >> bit) & 1) ? m : ~m;
    }
    const int rank = __popc(peers & lt);
    old[j] = 0;
    if (rr[j] >= 0 && rank == 0) old[j] = atomicAdd(&swh[w * R + rr[j]], __popc(peers));
    pk[j] = (uint32_t)(__ffs(peers) - 1) | ((uint32_t)rank << 5);
    __syncwarp();
  }
  __syncthreads();
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    int acc = base[(size_t)r * n_chunks + blockIdx.x];
    for (int q = 0; q < kScatterWarps; ++q) { const int c = swh[q * R + r]; swh[q * R + r] = acc; acc += c; }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kScatterPer; ++j) {
    const int o = __shfl_sync(0xffffffffu, old[j], (int)(pk[j] & 31u));
    if (rr[j] >= 0) {
      const int64_t p = s0 + j * 32 + lane;
      const int q = swh[w * R + rr[j]] + o + (int)(pk[j] >> 5);
      out[q] = tmp[p];
      uint32_t d = tmp_dep[p];
      if (order) {
        // the previous pairs of i and j lie in the same cell: the same shift
        const uint32_t sh = (uint32_t)(rr[j] - (tmp_round[p] & 0xFFFF));
        uint32_t di = d & 0xFFFFu, dj = d >> 16;
        if (di) di += sh;
        if (dj) dj += sh;
        d = di | (dj << 16);
      }
      deps[q] = d;
    }
  }
}

__global__ void k_sel_finalize(const int32_t* offs, int32_t n_cells, int64_t capacity,
                               const unsigned long long* n_cand, const int32_t* n_rounds,
                               dsmc_select_info_t* info) {
  const int64_t total = offs[n_cells];
  info->n_pairs = total;
  info->n_candidates = (int64_t)*n_cand;
  info->n_rounds = total > capacity ? 0 : *n_rounds;
  info->pad_ = 0;
}

// ---------------------------------------------------------------- workspace
struct SelWs {
  int32_t *counts, *offs, *tmp_round, *last, *round_count, *round_fill, *n_rounds;
  int32_t* chunk_cnt;  // [DSMC_MAX_ROUNDS][n_chunks] counts, then scatter bases
  int32_t n_chunks;
  int32_t *wcnt, *wofs, *ncand;
  uint32_t* bits;
  int64_t words_cap;
  uint32_t* tmp_dep;
  double* sgnew;
  int4* tmp;
  unsigned long long* n_cand;
  void* scan;
};

static size_t carve(SelWs* w, char* p, int32_t n, int32_t n_cells, int64_t capacity) {
  char* p0 = p;
  auto take = [&](size_t bytes) { char* q = p; p += align256(bytes); return q; };
  const size_t nc = (size_t)(n_cells > 0 ? n_cells : 1);
  const size_t cap = (size_t)(capacity > 0 ? capacity : 1);
  w->counts = (int32_t*)take(sizeof(int32_t) * nc);
  w->offs = (int32_t*)take(sizeof(int32_t) * (nc + 1));
  w->sgnew = (double*)take(sizeof(double) * nc);
  w->tmp = (int4*)take(sizeof(int4) * cap);
  w->tmp_round = (int32_t*)take(sizeof(int32_t) * cap);
  w->tmp_dep = (uint32_t*)take(sizeof(uint32_t) * cap);
  w->n_chunks = (int32_t)((cap + kScatterChunk - 1) / kScatterChunk);
  w->wcnt = (int32_t*)take(sizeof(int32_t) * nc);
  w->ncand = (int32_t*)take(sizeof(int32_t) * nc);
  w->wofs = (int32_t*)take(sizeof(int32_t) * (nc + 1));
  // accept bits for up to 32 candidates per accepted-pair slot
  w->words_cap = (int64_t)cap;
  w->bits = (uint32_t*)take(sizeof(uint32_t) * cap);
  w->chunk_cnt = (int32_t*)take(sizeof(int32_t) * (size_t)DSMC_MAX_ROUNDS * (size_t)w->n_chunks);
  w->last = (int32_t*)take(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  // the following four are zeroed together
  w->round_count = (int32_t*)take(sizeof(int32_t) * DSMC_MAX_ROUNDS * 2 + 256);
  w->round_fill = w->round_count + DSMC_MAX_ROUNDS;
  w->n_rounds = w->round_count + 2 * DSMC_MAX_ROUNDS;
  w->n_cand = (unsigned long long*)(w->round_count + 2 * DSMC_MAX_ROUNDS + 2);
  const size_t sws = scan_ws(n_cells) > scan_ws(DSMC_MAX_ROUNDS) ? scan_ws(n_cells) : scan_ws(DSMC_MAX_ROUNDS);
  w->scan = take(sws);
  return (size_t)(p - p0);
}

size_t select_ws(int32_t n, int32_t n_cells, int64_t capacity) {
  SelWs w;
  return carve(&w, (char*)0, n, n_cells, capacity);
}

static unsigned blocks_for(int64_t work, int per_block, int max_blocks) {
  int64_t b = (work + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (unsigned)b;
}

int launch_select(Ctx* c, const dsmc_gas_t& gas, int32_t n, int32_t n_cells, const int32_t* cs,
                  const double* vx, const double* vy, const double* vz, double* sgmax,
                  uint64_t step, int64_t capacity, int32_t* pairs, uint32_t* deps, int32_t* round_offsets,
                  dsmc_select_info_t* info, void* ws, size_t ws_bytes, int32_t order, cudaStream_t s) {
  if (ws_bytes < select_ws(n, n_cells, capacity))
    return record(c, DSMC_ERR_ARG, "select: workspace too small");
  if (capacity > INT32_MAX) return record(c, DSMC_ERR_ARG, "select: capacity >= 2^31");
  SelWs w;
  carve(&w, (char*)ws, n, n_cells, capacity);
  SelArgs a;
  a.cs = cs; a.vx = vx; a.vy = vy; a.vz = vz; a.sgmax = sgmax; a.sgnew = w.sgnew;
  a.counts = w.counts; a.offs = w.offs; a.tmp = w.tmp; a.tmp_round = w.tmp_round; a.tmp_dep = w.tmp_dep;
  a.wcnt = w.wcnt; a.wofs = w.wofs; a.bits = w.bits; a.words_cap = w.words_cap; a.ncand = w.ncand;
  a.last = w.last; a.round_count = w.round_count; a.n_rounds = w.n_rounds; a.n_cand = w.n_cand;
  a.status = status_ptr(c); a.n_cells = n_cells; a.capacity = capacity;
  a.seed = gas.seed; a.key = philox_key(gas.seed); a.step = step; a.step_dev = graph_step_ptr(c); a.fn = gas.fn_over_vc; a.dt = gas.dt;
  sel_model(a, gas);
  a.order = order;
  const int sms = sm_count(c);
  if (cudaMemsetAsync(w.round_count, 0, sizeof(int32_t) * DSMC_MAX_ROUNDS * 2 + 256, s) != cudaSuccess)
    return DSMC_ERR_CUDA;
  if (cudaMemsetAsync(round_offsets, 0, sizeof(int32_t) * (DSMC_MAX_ROUNDS + 1), s) != cudaSuccess)
    return DSMC_ERR_CUDA;
  if (n_cells > 0) {
    k_sel_nwords<<<blocks_for(n_cells, 256, sms * 4), 256, 0, s>>>(a);
    count_launches(c, 1);
    int rcw = launch_scan(c, w.wcnt, w.wofs, n_cells, w.scan, s);
    if (rcw) return rcw;
    const unsigned gb = blocks_for((n_cells + 1) / 2, kSelWarps, sms * 8);
    k_sel_count<<<gb, kSelWarps * 32, 0, s>>>(a);
    count_launches(c, 1);
    int rc = launch_scan(c, w.counts, w.offs, n_cells, w.scan, s);
    if (rc) return rc;
    k_sel_emit<<<blocks_for((n_cells + 1) / 2, kEmitWarps, sms * 16), kEmitWarps * 32, 0, s>>>(a);
    count_launches(c, 1);
    // at least one block: the capacity-overflow commit of (sigma g)_max runs in k_sel_rcount
    const unsigned sb = (unsigned)((capacity + kScatterChunk - 1) / kScatterChunk) + (capacity <= 0);
    {
      k_sel_rcount<<<sb, 256, 0, s>>>(w.tmp_round, w.offs, n_cells, capacity, w.n_rounds, w.n_chunks, w.chunk_cnt,
                                      w.sgnew, sgmax, order, w.round_count);
      k_sel_rscan<<<DSMC_MAX_ROUNDS, 256, 0, s>>>(w.offs, n_cells, capacity, w.n_rounds, w.round_count,
                                                 round_offsets, w.n_chunks, w.chunk_cnt);
      const int ssm = (int)(sizeof(int) * kScatterWarps * DSMC_MAX_ROUNDS);
      if (cudaFuncSetAttribute(k_sel_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, ssm) != cudaSuccess)
        return DSMC_ERR_CUDA;
      k_sel_scatter<<<sb, kScatterWarps * 32, ssm, s>>>(w.tmp, w.tmp_round, w.tmp_dep, w.offs, n_cells, capacity,
                                                       w.n_rounds, w.n_chunks, w.chunk_cnt, (int4*)pairs, deps,
                                                       order);
      count_launches(c, 3);
    }
  } else {
    if (cudaMemsetAsync(w.offs, 0, sizeof(int32_t), s) != cudaSuccess) return DSMC_ERR_CUDA;
  }
  k_sel_finalize<<<1, 1, 0, s>>>(w.offs, n_cells, capacity, w.n_cand, w.n_rounds, info);
  count_launches(c, 1);
  return cudaGetLastError() == cudaSuccess ? 0 : DSMC_ERR_CUDA;
}

// ---------------------------------------------------------------- (sigma g)_max init
__global__ void k_sgmax_init(SelArgs a, const double* T, double factor, double mass, double* out) {
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < a.n_cells; k += gridDim.x * blockDim.x) {
    const double g0 = factor * sqrt(2.0 * DSMC_KB * T[k] / mass);
    out[k] = sigma_g(a, g0);
  }
}

int launch_sgmax_init(Ctx* c, const dsmc_gas_t& gas, int32_t n_cells, const double* T,
                      double factor, double* sgmax, cudaStream_t s) {
  if (n_cells <= 0) return 0;
  SelArgs a = {};
  a.n_cells = n_cells;
  sel_model(a, gas);
  k_sgmax_init<<<blocks_for(n_cells, 256, sm_count(c) * 4), 256, 0, s>>>(a, T, factor, gas.mass, sgmax);
  count_launches(c, 1);
  return cudaGetLastError() == cudaSuccess ? 0 : DSMC_ERR_CUDA;
}

}  // namespace dsmc
