// Cell sort, cell moments, moment matching and the int32 exclusive scan.
//
// Sort (Sec. 2.6 (1)): a stable LSD radix sort of (cell id, input index) on
// 9-bit digits (two passes for up to 2^18 cells), each pass a per-chunk
// digit count, one exclusive scan over (digit, chunk) and an ordered
// per-chunk scatter; cell_start from the sorted ids; then the gather of the
// velocities.  (The allocation-free variant keeps an atomic histogram +
// cursor scatter + per-cell sort of the slots.)  Moments and moment
// matching use exact integer sums over 8 lanes per cell (moments.cuh).
#include <climits>

#include "internal.cuh"
#include "moments.cuh"

namespace dsmc {

// ---------------------------------------------------------------- scan
// Reduce-then-scan over blocks of kScanItems elements.
constexpr int kScanThreads = 256;
constexpr int kScanPer = 16;
constexpr int kScanItems = kScanThreads * kScanPer;

__device__ __forceinline__ int block_exclusive_scan(int v, int* total) {
  __shared__ int wsum[kScanThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int s = lane < kScanThreads / 32 ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < kScanThreads / 32) wsum[lane] = s;
  }
  __syncthreads();
  const int before = (wid ? wsum[wid - 1] : 0) + x - v;
  *total = wsum[kScanThreads / 32 - 1];
  __syncthreads();
  return before;
}

__global__ void k_scan_reduce(const int32_t* __restrict__ in, int64_t n, int32_t* bsum) {
  const int64_t base = (int64_t)blockIdx.x * kScanItems;
  int s = 0;
  for (int q = 0; q < kScanPer; ++q) {
    const int64_t i = base + (int64_t)q * kScanThreads + threadIdx.x;
    if (i < n) s += in[i];
  }
  int total;
  block_exclusive_scan(s, &total);
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void k_scan_blocks(int32_t* bsum, int64_t nb) {
  int carry = 0;
  for (int64_t b0 = 0; b0 < nb; b0 += kScanThreads) {
    const int64_t i = b0 + threadIdx.x;
    const int v = i < nb ? bsum[i] : 0;
    int total;
    const int ex = block_exclusive_scan(v, &total);
    if (i < nb) bsum[i] = carry + ex;
    carry += total;
  }
}

__global__ void k_scan_apply(const int32_t* __restrict__ in, int64_t n, const int32_t* bsum,
                             int32_t* __restrict__ out) {
  const int64_t base = (int64_t)blockIdx.x * kScanItems + (int64_t)threadIdx.x * kScanPer;
  int v[kScanPer];
  int s = 0;
#pragma unroll
  for (int q = 0; q < kScanPer; ++q) {
    v[q] = base + q < n ? in[base + q] : 0;
    s += v[q];
  }
  int total;
  int run = bsum[blockIdx.x] + block_exclusive_scan(s, &total);
#pragma unroll
  for (int q = 0; q < kScanPer; ++q) {
    if (base + q < n) out[base + q] = run;
    run += v[q];
  }
  if (base <= n - 1 && n - 1 < base + kScanPer) out[n] = run;  // total after the last element
}

size_t scan_ws(int64_t n) { return align256(sizeof(int32_t) * (size_t)((n + kScanItems - 1) / kScanItems + 1)); }

int launch_scan(Ctx* c, const int32_t* in, int32_t* out, int64_t n, void* ws, cudaStream_t s) {
  if (n <= 0) {
    return cudaMemsetAsync(out, 0, sizeof(int32_t), s) == cudaSuccess ? 0 : DSMC_ERR_CUDA;
  }
  const int64_t nb = (n + kScanItems - 1) / kScanItems;
  int32_t* bsum = (int32_t*)ws;
  k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, bsum);
  k_scan_blocks<<<1, kScanThreads, 0, s>>>(bsum, nb);
  k_scan_apply<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, bsum, out);
  if (c) count_launches(c, 3);
  return cudaGetLastError() == cudaSuccess ? 0 : DSMC_ERR_CUDA;
}

// ---------------------------------------------------------------- sort
__global__ void k_hist(const int32_t* __restrict__ cell_id, int32_t n, int32_t n_cells,
                       int32_t* counts, int* status) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int32_t c = cell_id[i];
    if ((uint32_t)c < (uint32_t)n_cells) atomicAdd(counts + c, 1);
    else set_status(status, DSMC_ERR_ARG);
  }
}

__global__ void k_scatter(const int32_t* __restrict__ cell_id, int32_t n, int32_t n_cells,
                          const int32_t* __restrict__ cell_start, int32_t* fill,
                          int32_t* __restrict__ slots) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int32_t c = cell_id[i];
    if ((uint32_t)c >= (uint32_t)n_cells) continue;
    slots[cell_start[c] + atomicAdd(fill + c, 1)] = i;
  }
}

constexpr int kFixWarps = 8;
constexpr int kFixCap = 1024;  // cells up to this size sort in shared memory, one warp each

// Warp per cell of at most kFixCap particles: order the cell's slot contents
// ascending (bitonic network in shared memory).  Larger cells are left to
// k_fix_large.
__global__ void __launch_bounds__(kFixWarps * 32)
k_fix_gather(int32_t n_cells, const int32_t* __restrict__ cell_start,
             const int32_t* __restrict__ slots, int32_t* __restrict__ perm) {
  __shared__ int buf_all[kFixWarps][kFixCap];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int* buf = buf_all[wid];
  const int32_t warps = gridDim.x * kFixWarps;
  for (int32_t k = blockIdx.x * kFixWarps + wid; k < n_cells; k += warps) {
    const int32_t a = cell_start[k], N = cell_start[k + 1] - a;
    if (N <= 0) continue;
    if (N <= kFixCap) {
      int P = 1;
      while (P < N) P <<= 1;
      for (int t = lane; t < P; t += 32) buf[t] = t < N ? slots[a + t] : INT_MAX;
      __syncwarp();
      for (int kk = 2; kk <= P; kk <<= 1) {
        for (int j = kk >> 1; j > 0; j >>= 1) {
          for (int t = lane; t < (P >> 1); t += 32) {
            const int i = (t / j) * 2 * j + (t % j);
            const int ixj = i + j;
            const int x = buf[i], y = buf[ixj];
            const bool up = (i & kk) == 0;
            if ((x > y) == up) { buf[i] = y; buf[ixj] = x; }
          }
          __syncwarp();
        }
      }
      for (int t = lane; t < N; t += 32) perm[a + t] = buf[t];
    }
  }
}

// Block per cell of more than kFixCap particles: the cell's slot contents
// (distinct input indices below 2^24) sorted ascending by a stable LSD radix
// sort on 8-bit digits, three passes that alternate between the cell's slot
// range (scratch) and its perm range: slots -> perm -> slots -> perm.  Each
// pass counts the digits of the whole cell, then scatters it in order in
// tiles of kLgTile values: warp w of the block owns the tile's w-th
// segment (kLgPer values per lane, in order), the warps' digit counts become
// per-warp starting positions, and equal digits within a warp are ranked by
// lane from ballots.  O(N) work per cell; a cell of 2^20 particles takes
// 3 x 256 tiles.
constexpr int kLgWarps = 16;
constexpr int kLgPer = 8;
constexpr int kLgTile = kLgWarps * 32 * kLgPer;
constexpr int kLgBits = 8;
constexpr int kLgRadix = 1 << kLgBits;

__global__ void __launch_bounds__(kLgWarps * 32)
k_fix_large(int32_t n_cells, const int32_t* __restrict__ cell_start, int32_t* slots, int32_t* perm) {
  __shared__ int run[kLgRadix];               // the cell's digit counts, then running positions
  __shared__ int wh[kLgWarps][kLgRadix];      // per-warp positions inside the current tile
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  for (int32_t k = blockIdx.x; k < n_cells; k += gridDim.x) {
    const int32_t a = cell_start[k], N = cell_start[k + 1] - a;
    if (N <= kFixCap) continue;
    for (int pass = 0; pass < 3; ++pass) {
      const int32_t* src = (pass & 1) ? perm + a : slots + a;
      int32_t* dst = (pass & 1) ? slots + a : perm + a;
      const int shift = pass * kLgBits;
      for (int t = threadIdx.x; t < kLgRadix; t += blockDim.x) run[t] = 0;
      __syncthreads();
      for (int32_t t = threadIdx.x; t < N; t += blockDim.x) atomicAdd(&run[(src[t] >> shift) & (kLgRadix - 1)], 1);
      __syncthreads();
      if (w == 0) {   // exclusive scan of the 256 counts, 8 per lane
        int c[kLgRadix / 32], sum = 0;
#pragma unroll
        for (int q = 0; q < kLgRadix / 32; ++q) { c[q] = run[lane * (kLgRadix / 32) + q]; sum += c[q]; }
        int x = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, x, o);
          if (lane >= o) x += y;
        }
        int acc = x - sum;
#pragma unroll
        for (int q = 0; q < kLgRadix / 32; ++q) { run[lane * (kLgRadix / 32) + q] = acc; acc += c[q]; }
      }
      __syncthreads();
      for (int32_t t0 = 0; t0 < N; t0 += kLgTile) {
        const int32_t s0 = t0 + w * (32 * kLgPer);
        int32_t val[kLgPer];
#pragma unroll
        for (int j = 0; j < kLgPer; ++j) {
          const int32_t i = s0 + j * 32 + lane;
          val[j] = i < N ? src[i] : -1;
        }
        for (int t = threadIdx.x; t < kLgWarps * kLgRadix; t += blockDim.x) wh[t / kLgRadix][t % kLgRadix] = 0;
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kLgPer; ++j)
          if (val[j] >= 0) atomicAdd(&wh[w][(val[j] >> shift) & (kLgRadix - 1)], 1);
        __syncthreads();
        for (int d = threadIdx.x; d < kLgRadix; d += blockDim.x) {
          int acc = run[d];
          for (int q = 0; q < kLgWarps; ++q) { const int c = wh[q][d]; wh[q][d] = acc; acc += c; }
          run[d] = acc;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kLgPer; ++j) {
          const bool has = val[j] >= 0;
          const int d = has ? (val[j] >> shift) & (kLgRadix - 1) : -1;
          // lanes with the same digit (lanes without a value form their own set)
          unsigned same = __ballot_sync(0xffffffffu, has);
          if (!has) same = ~same;
#pragma unroll
          for (int bit = 0; bit < kLgBits; ++bit) {
            const unsigned m = __ballot_sync(0xffffffffu, (d >> bit) & 1);
            same &= ((d >> bit) & 1) ? m : ~m;
          }
          if (has) dst[wh[w][d] + __popc(same & lt)] = val[j];
          __syncwarp();
          if (has && (same & lt) == 0) wh[w][d] += __popc(same);
          __syncwarp();
        }
        __syncthreads();
      }
    }
  }
}

// Thread per sorted slot: gather the velocities (independent random loads).
// Only the cell_start[n_cells] slots that the scatter filled are read: a
// particle with an out-of-range cell id (reported as DSMC_ERR_ARG) has no
// slot, and the perm entries past the filled ones are never written.
__global__ void k_gather(int32_t n, const int32_t* __restrict__ cell_start, int32_t n_cells,
                         const int32_t* __restrict__ perm, const double* __restrict__ vx,
                         const double* __restrict__ vy, const double* __restrict__ vz,
                         double* __restrict__ svx, double* __restrict__ svy, double* __restrict__ svz) {
  const int32_t filled = min(n, cell_start[n_cells]);
  // four slots per thread per pass, their loads issued before any store, so
  // that twelve independent random reads per thread are in flight
  constexpr int kIlp = 4;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t s0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s0 < filled; s0 += kIlp * stride) {
    int32_t src[kIlp];
#pragma unroll
    for (int u = 0; u < kIlp; ++u) {
      const int64_t s = s0 + u * stride;
      src[u] = s < filled ? __ldcs(perm + s) : -1;
    }
    double x[kIlp], y[kIlp], z[kIlp];
#pragma unroll
    for (int u = 0; u < kIlp; ++u) {
      if (src[u] >= 0) { x[u] = __ldg(vx + src[u]); y[u] = __ldg(vy + src[u]); z[u] = __ldg(vz + src[u]); }
    }
#pragma unroll
    for (int u = 0; u < kIlp; ++u) {
      const int64_t s = s0 + u * stride;
      if (src[u] >= 0) { svx[s] = x[u]; svy[s] = y[u]; svz[s] = z[u]; }
    }
  }
}

// One velocity component at a time: the 73 MB source array of a 9M-particle
// gas stays in L2 (129 MB) while its random reads land, so each sector comes
// from DRAM once instead of once per particle that reads it.  perm and the
// output stream through with evict-first hints so that they do not push
// the source array out.
__global__ void k_gather1(int32_t n, const int32_t* __restrict__ cell_start, int32_t n_cells,
                          const int32_t* __restrict__ perm, const double* __restrict__ v,
                          double* __restrict__ sv) {
  const int32_t filled = min(n, cell_start[n_cells]);
  constexpr int kIlp = 4;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t s0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s0 < filled; s0 += kIlp * stride) {
    int32_t src[kIlp];
#pragma unroll
    for (int u = 0; u < kIlp; ++u) {
      const int64_t s = s0 + u * stride;
      src[u] = s < filled ? __ldcs(perm + s) : -1;
    }
    double x[kIlp];
#pragma unroll
    for (int u = 0; u < kIlp; ++u)
      if (src[u] >= 0) x[u] = __ldg(v + src[u]);
#pragma unroll
    for (int u = 0; u < kIlp; ++u)
      if (src[u] >= 0) __stcs(sv + s0 + u * stride, x[u]);
  }
}

// ---------------------------------------------------------------- radix sort
constexpr int kRadixBits = 9;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kRsChunk = 4096;   // elements per block
constexpr int kRsWarps = 16;

// key of input element i: its cell id, or n_cells for an id out of range
// (recorded as DSMC_ERR_ARG; such particles sort after every cell)
__device__ __forceinline__ uint32_t rs_key(const int32_t* cell_id, const uint32_t* keys, int64_t i,
                                           int32_t n_cells, int* status) {
  if (keys) return keys[i];
  const int32_t c = cell_id[i];
  if ((uint32_t)c < (uint32_t)n_cells) return (uint32_t)c;
  if (status) set_status(status, DSMC_ERR_ARG);
  return (uint32_t)n_cells;
}

// cnt[d * chunks + block] = elements of the block's chunk with digit d
__global__ void __launch_bounds__(256)
k_rs_count(const int32_t* __restrict__ cell_id, const uint32_t* __restrict__ keys, int32_t n, int32_t n_cells,
           int shift, int32_t chunks, int32_t* __restrict__ cnt, int* status) {
  __shared__ int hist[kRadix];
  for (int t = threadIdx.x; t < kRadix; t += blockDim.x) hist[t] = 0;
  __syncthreads();
  const int64_t p0 = (int64_t)blockIdx.x * kRsChunk, p1 = min((int64_t)n, p0 + kRsChunk);
  for (int64_t i = p0 + threadIdx.x; i < p1; i += blockDim.x)
    atomicAdd(&hist[(rs_key(cell_id, keys, i, n_cells, status) >> shift) & (kRadix - 1)], 1);
  __syncthreads();
  for (int t = threadIdx.x; t < kRadix; t += blockDim.x) cnt[(size_t)t * chunks + blockIdx.x] = hist[t];
}

// Block d: exclusive scan of digit d's counts over the chunks (row d of
// the digit-major table, in place into off) and the digit's total.
__global__ void __launch_bounds__(256)
k_rs_rowscan(const int32_t* __restrict__ cnt, int32_t chunks, int32_t* __restrict__ off, int32_t* __restrict__ tot) {
  __shared__ int wt[8];
  __shared__ int carry;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int32_t* row = cnt + (size_t)blockIdx.x * chunks;
  int32_t* orow = off + (size_t)blockIdx.x * chunks;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int32_t c0 = 0; c0 < chunks; c0 += 256) {
    const int32_t c = c0 + threadIdx.x;
    const int v = c < chunks ? row[c] : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wt[w] = x;
    __syncthreads();
    int before = carry;
    for (int q = 0; q < w; ++q) before += wt[q];
    if (c < chunks) orow[c] = before + x - v;
    __syncthreads();
    if (threadIdx.x == 255) carry = before + x;
    __syncthreads();
  }
  if (threadIdx.x == 0) tot[blockIdx.x] = carry;
}

// Ordered scatter of one chunk: warp w owns the chunk's w-th sixteenth, its
// kRsPer elements per lane loaded into registers first.  Stable ranks in
// two steps: (1) per element batch j (32 consecutive elements), the lanes
// holding the same digit find each other from one ballot per digit bit; the lowest
// of them adds the group's size to the warp's counter of that digit in
// shared memory and keeps the old value (the count of that digit in the
// warp's earlier batches; the batches' atomics are ordered by __syncwarp),
// the others their rank inside the group.  (2) After the counts are
// complete, each counter becomes the warp's starting position for its digit
// in the chunk's own digit order (the digit's start in the chunk, then the
// warps in order), and every element's place is that warp start + old
// value of its group's leader + rank.  No element waits on the
// shared-memory result of the batch before it.  (3) The chunk is reordered
// by digit in shared memory and written out from there: consecutive threads
// write consecutive addresses of each digit's run (its global start from
// the scan), so the stores coalesce.
// Values: the input index (first pass) or vals.
constexpr int kRsPer = kRsChunk / kRsWarps / 32;
static_assert(kRsWarps * 32 == kRadix, "one thread per digit in the offset step");

__global__ void __launch_bounds__(kRsWarps * 32, 2)
k_rs_scatter(const int32_t* __restrict__ cell_id, const uint32_t* __restrict__ keys,
             const int32_t* __restrict__ vals, int32_t n, int32_t n_cells, int shift, int32_t chunks,
             const int32_t* __restrict__ base, const int32_t* __restrict__ tot, uint32_t* __restrict__ keys_out,
             int32_t* __restrict__ vals_out) {
  __shared__ union {
    int wh[kRsWarps][kRadix];                              // per-warp digit counters, then positions
    struct { uint32_t key[kRsChunk]; int32_t val[kRsChunk]; } st;  // the chunk in digit order
  } sm;
  __shared__ int gdelta[kRadix];   // global start - chunk-local start of each digit
  __shared__ int wt[kRsWarps], wg[kRsWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < kRsWarps * kRadix; t += blockDim.x) sm.wh[t / kRadix][t % kRadix] = 0;
  // 32-bit unsigned indices (below n + 4096 < 2^32)
  const uint32_t un = (uint32_t)n;
  const uint32_t c0 = blockIdx.x * (uint32_t)kRsChunk;
  const uint32_t s0 = c0 + (uint32_t)w * (kRsPer * 32);
  uint32_t key[kRsPer];
  int32_t val[kRsPer];
#pragma unroll
  for (int j = 0; j < kRsPer; ++j) {
    const uint32_t i = s0 + j * 32 + lane;
    const bool has = i < un;
    key[j] = has ? rs_key(cell_id, keys, i, n_cells, nullptr) : 0u;
    val[j] = has ? (vals ? vals[i] : (int32_t)i) : 0;
  }
  __syncthreads();
  const unsigned lt = (1u << lane) - 1u;
  int old[kRsPer];
  uint32_t pk[kRsPer];   // leader lane | rank in the group << 5
#pragma unroll
  for (int j = 0; j < kRsPer; ++j) {
    const bool has = s0 + j * 32 + lane < un;
    // lanes without an element share the digit kRadix (no counter)
    const int d = has ? (int)((key[j] >> shift) & (kRadix - 1)) : kRadix;
    // lanes holding the same digit: one ballot per digit bit (ALU pipe); the
    // lanes without an element form their own set
    unsigned peers = __ballot_sync(0xffffffffu, has);
    if (!has) peers = ~peers;
#pragma unroll
    for (int bit = 0; bit < kRadixBits; ++bit) {
      const unsigned m = __ballot_sync(0xffffffffu, (d >> bit) & 1);
      peers &= ((d >> bit) & 1) ? m : ~m;
    }
    const int rank = __popc(peers & lt);
    old[j] = 0;
    if (has && rank == 0) old[j] = atomicAdd(&sm.wh[w][d], __popc(peers));
    pk[j] = (uint32_t)(__ffs(peers) - 1) | ((uint32_t)rank << 5);
    __syncwarp();
  }
  __syncthreads();
  {
    // thread d: the warps' positions for digit d inside the chunk's digit
    // order (exclusive scan of the digit totals, then the warps in order)
    // (and the digit's global start: the totals of the smaller digits plus
    // the digit's count in earlier chunks)
    const int d = threadIdx.x;
    int ct = 0;
#pragma unroll
    for (int q = 0; q < kRsWarps; ++q) ct += sm.wh[q][d];
    const int gt = tot[d];
    int x = ct, xg = gt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o), yg = __shfl_up_sync(0xffffffffu, xg, o);
      if (lane >= o) { x += y; xg += yg; }
    }
    if (lane == 31) { wt[w] = x; wg[w] = xg; }
    __syncthreads();
    if (w == 0) {
      int v = lane < kRsWarps ? wt[lane] : 0, vg = lane < kRsWarps ? wg[lane] : 0;
#pragma unroll
      for (int o = 1; o < kRsWarps; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, o), yg = __shfl_up_sync(0xffffffffu, vg, o);
        if (lane >= o) { v += y; vg += yg; }
      }
      if (lane < kRsWarps) { wt[lane] = v; wg[lane] = vg; }
    }
    __syncthreads();
    const int ls = (w ? wt[w - 1] : 0) + x - ct;    // chunk-local start of digit d
    const int gs = (w ? wg[w - 1] : 0) + xg - gt;   // global start of digit d
    gdelta[d] = gs + base[(size_t)d * chunks + blockIdx.x] - ls;
    int acc = ls;
#pragma unroll
    for (int q = 0; q < kRsWarps; ++q) { const int c = sm.wh[q][d]; sm.wh[q][d] = acc; acc += c; }
  }
  __syncthreads();
  int lp[kRsPer];
#pragma unroll
  for (int j = 0; j < kRsPer; ++j) {
    const int o = __shfl_sync(0xffffffffu, old[j], (int)(pk[j] & 31u));
    const int d = (int)((key[j] >> shift) & (kRadix - 1));
    lp[j] = sm.wh[w][d] + o + (int)(pk[j] >> 5);
  }
  __syncthreads();   // every position read before the counters' storage is reused
#pragma unroll
  for (int j = 0; j < kRsPer; ++j) {
    if (s0 + j * 32 + lane < un) { sm.st.key[lp[j]] = key[j]; sm.st.val[lp[j]] = val[j]; }
  }
  __syncthreads();
  const int cnt = (int)min((uint32_t)kRsChunk, un - c0);
  for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
    const uint32_t k = sm.st.key[t];
    const int q = t + gdelta[(k >> shift) & (kRadix - 1)];
    if (keys_out) keys_out[q] = k;
    vals_out[q] = sm.st.val[t];
  }
}

// cell_start from the sorted keys: slot s starts every cell in (key[s-1], key[s]]
// (slot n closes the list with key n_cells).  Four slots per thread.
__global__ void k_cell_start(const uint32_t* __restrict__ skeys, int32_t n, int32_t n_cells,
                             int32_t* __restrict__ cell_start) {
  // 32-bit indices: slots 0..n (n < 2^31), keys 0..n_cells
  const uint32_t un = (uint32_t)n, stride = gridDim.x * blockDim.x * 4u;
  for (uint32_t s0 = (blockIdx.x * blockDim.x + threadIdx.x) * 4u; s0 <= un; s0 += stride) {
    int32_t key[5];   // key[q] = skeys[s0 - 1 + q] (-1 before the first slot, n_cells from slot n on)
    key[0] = s0 > 0 ? (int32_t)skeys[s0 - 1] : -1;
    if (s0 + 4 <= un && ((uintptr_t)(skeys + s0) & 15) == 0) {
      const uint4 k4 = __ldcs(reinterpret_cast<const uint4*>(skeys + s0));
      key[1] = (int32_t)k4.x; key[2] = (int32_t)k4.y; key[3] = (int32_t)k4.z; key[4] = (int32_t)k4.w;
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) key[q + 1] = s0 + q < un ? (int32_t)skeys[s0 + q] : n_cells;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t s = s0 + q;
      if (s > un) break;
      for (int32_t c = key[q] + 1; c <= key[q + 1] && c <= n_cells; ++c) cell_start[c] = (int32_t)s;
    }
  }
}

static int radix_passes(int32_t n_cells) {
  int bits = 1;
  while (bits < 31 && ((int64_t)1 << bits) <= (int64_t)n_cells) ++bits;  // keys up to n_cells
  return (bits + kRadixBits - 1) / kRadixBits;
}

size_t sort_ws(int32_t n, int32_t n_cells) {
  const size_t nn = (size_t)(n > 0 ? n : 1);
  const size_t chunks = (nn + kRsChunk - 1) / kRsChunk;
  const size_t tab = (size_t)kRadix * chunks;
  return 4 * align256(sizeof(uint32_t) * nn)        // keys and values, two buffers each
         + 2 * align256(sizeof(int32_t) * (tab + 1)) // digit counts and their scan along the chunks
         + align256(sizeof(int32_t) * kRadix);       // digit totals
}

static unsigned grid_for(int64_t work, int per_block, int max_blocks) {
  int64_t b = (work + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (unsigned)b;
}

int launch_sort(Ctx* c, int32_t n, int32_t n_cells, const int32_t* cell_id, const double* vx,
                const double* vy, const double* vz, int32_t* perm, int32_t* cell_start,
                double* svx, double* svy, double* svz, void* ws, size_t ws_bytes,
                cudaStream_t s) {
  if (int rc = launch_sort_keys(c, n, n_cells, cell_id, perm, cell_start, ws, ws_bytes, s)) return rc;
  return launch_gather(c, n, n_cells, cell_start, perm, vx, vy, vz, svx, svy, svz, s);
}

// The radix passes on the cell ids alone: perm and cell_start (the velocities
// are not read, so their upload may still be in flight).
int launch_sort_keys(Ctx* c, int32_t n, int32_t n_cells, const int32_t* cell_id, int32_t* perm,
                     int32_t* cell_start, void* ws, size_t ws_bytes, cudaStream_t s) {
  if (ws_bytes < sort_ws(n, n_cells)) return record(c, DSMC_ERR_ARG, "sort: workspace too small");
  const size_t nn = (size_t)(n > 0 ? n : 1);
  const int32_t chunks = (int32_t)((nn + kRsChunk - 1) / kRsChunk);
  const size_t tab = (size_t)kRadix * chunks;
  char* p = (char*)ws;
  auto take = [&](size_t bytes) { char* q = p; p += align256(bytes); return q; };
  uint32_t* ka = (uint32_t*)take(4 * nn);
  int32_t* va = (int32_t*)take(4 * nn);
  uint32_t* kb = (uint32_t*)take(4 * nn);
  int32_t* vb = (int32_t*)take(4 * nn);
  int32_t* cnt = (int32_t*)take(4 * (tab + 1));
  int32_t* off = (int32_t*)take(4 * (tab + 1));
  int32_t* dtot = (int32_t*)take(sizeof(int32_t) * kRadix);   // digit totals
  if (n == 0) {
    k_cell_start<<<1, 256, 0, s>>>(kb, 0, n_cells, cell_start);
    count_launches(c, 1);
    return cudaGetLastError() == cudaSuccess ? 0 : DSMC_ERR_CUDA;
  }
  const int passes = radix_passes(n_cells);
  const uint32_t* kin = nullptr;   // first pass: keys from cell_id
  const int32_t* vin = nullptr;    // first pass: values = input index
  for (int q = 0; q < passes; ++q) {
    const bool last = q + 1 == passes;
    uint32_t* kout = (q & 1) ? kb : ka;
    int32_t* vout = last ? perm : ((q & 1) ? vb : va);
    k_rs_count<<<chunks, 256, 0, s>>>(cell_id, kin, n, n_cells, q * kRadixBits, chunks, cnt,
                                      q == 0 ? status_ptr(c) : nullptr);
    count_launches(c, 1);
    k_rs_rowscan<<<kRadix, 256, 0, s>>>(cnt, chunks, off, dtot);
    k_rs_scatter<<<chunks, kRsWarps * 32, 0, s>>>(cell_id, kin, vin, n, n_cells, q * kRadixBits, chunks, off,
                                                  dtot, kout, vout);
    count_launches(c, 2);
    kin = kout;
    vin = vout;
  }
  k_cell_start<<<grid_for(((int64_t)n + 4) / 4, 256, sm_count(c) * 8), 256, 0, s>>>(kin, n, n_cells, cell_start);
  count_launches(c, 1);
  return cudaGetLastError() == cudaSuccess ? 0 : DSMC_ERR_CUDA;
}

// one component: sv[s] = v[perm[s]]
int launch_gather_one(Ctx* c, int32_t n, int32_t n_cells, const int32_t* cell_start, const int32_t* perm,
                      const double* v, double* sv, cudaStream_t s) {
  if (n <= 0) return 0;
  const Shape sh = shape_or_default(c, DSMC_TUNE_GATHER);
  const unsigned g = grid_for(n, sh.threads, sm_count(c) * sh.blocks_per_sm);
  k_gather1<<<g, sh.threads, 0, s>>>(n, cell_start, n_cells, perm, v, sv);
  count_launches(c, 1);
  return cudaGetLastError() == cudaSuccess ? 0 : DSMC_ERR_CUDA;
}

int launch_gather(Ctx* c, int32_t n, int32_t n_cells, const int32_t* cell_start, const int32_t* perm,
                  const double* vx, const double* vy, const double* vz, double* svx, double* svy,
                  double* svz, cudaStream_t s) {
  if (n <= 0) return 0;
  const Shape sh = shape_or_default(c, DSMC_TUNE_GATHER);
  const unsigned g = grid_for(n, sh.threads, sm_count(c) * sh.blocks_per_sm);
  k_gather1<<<g, sh.threads, 0, s>>>(n, cell_start, n_cells, perm, vx, svx);
  k_gather1<<<g, sh.threads, 0, s>>>(n, cell_start, n_cells, perm, vy, svy);
  k_gather1<<<g, sh.threads, 0, s>>>(n, cell_start, n_cells, perm, vz, svz);
  count_launches(c, 3);
  return cudaGetLastError() == cudaSuccess ? 0 : DSMC_ERR_CUDA;
}

// ---------------------------------------------------------------- moments
// Cell moments and moment matching without block-wide synchronisation: each
// warp claims runs of kCwRun consecutive cells from a counter (so that the
// warps given cheap runs, such as empty cells or the free stream, take more
// of them) and collects kCwClaims runs before finishing their cells.
// Segments of 8 lanes take four cells at a time through the two passes of
// the exact integer moments (the largest exponent, then the split sums of
// moments.cuh); the per-cell remainder (means, centred sum of squares,
// FP64 results) then runs one lane per cell, so that its FP64 instructions
// serve 16 cells at once; moment matching finally updates each run's
// particles one lane per particle, four at a time (three FP64 FMAs each,
// every lane busy, coalesced reads and writes).
constexpr int kCwWarps = 8;
constexpr int kCwRun = 8;                    // cells per claim
constexpr int kCwClaims = 2;                 // claims per batch
constexpr int kCwCells = kCwRun * kCwClaims; // cells per batch (one lane each in the remainder)

struct CwWarp {
  FixAcc acc[kCwCells];
  int E[kCwCells];
  int32_t cs[kCwClaims][kCwRun + 1];
  int32_t k0[kCwClaims];
  double coef[kCwCells][4];   // alpha and the three offsets (moment matching)
};

template <int SEG>
__device__ __forceinline__ FixAcc seg_sum_acc(FixAcc q) {
  q.sx = seg_sum_ll<SEG>(q.sx); q.sy = seg_sum_ll<SEG>(q.sy); q.sz = seg_sum_ll<SEG>(q.sz);
  q.A = (unsigned long long)seg_sum_ll<SEG>((long long)q.A);
  q.B = (unsigned long long)seg_sum_ll<SEG>((long long)q.B);
  q.L = (unsigned long long)seg_sum_ll<SEG>((long long)q.L);
  return q;
}

// Sums of one cell [a, b) by the SEG lanes of a segment (lane sl); returns
// the segment-reduced sums and *E.  Called by whole warps (lanes of a
// segment without a cell pass an empty range).
template <int SEG>
__device__ __forceinline__ FixAcc cell_sums(const double* __restrict__ X, const double* __restrict__ Y,
                                            const double* __restrict__ Z, int32_t a, int32_t b, int sl, int* E_out) {
  int E = 0;
#pragma unroll 4
  for (int32_t i = a + sl; i < b; i += SEG) E = max(E, max(dexp(X[i]), max(dexp(Y[i]), dexp(Z[i]))));
  E = seg_max_i<SEG>(E);
  const int32_t n = b - a;
  const int Ec = E + cell_scale(E, n).c, sp = fix_split(n);
  FixAcc q{0, 0, 0, 0ull, 0ull, 0ull};
#pragma unroll 4
  for (int32_t i = a + sl; i < b; i += SEG) {
    fix_add(q, q.sx, X[i], Ec, sp);
    fix_add(q, q.sy, Y[i], Ec, sp);
    fix_add(q, q.sz, Z[i], Ec, sp);
  }
  *E_out = E;
  return seg_sum_acc<SEG>(q);
}

// v <- alpha v + o over the particles [p0, p1) of one run of cells (cell
// starts cs[0..nc]), coefficients coef[0..nc); four particles per lane at
// a time, their loads issued together.
__device__ __forceinline__ void apply_run(const int32_t* cs, int nc, const double (*coef)[4], double* vx, double* vy,
                                          double* vz) {
  const int lane = threadIdx.x & 31;
  const int32_t p0 = cs[0], p1 = cs[nc];
  int c = 0;
  for (int32_t pb = p0; pb < p1; pb += 128) {
    double x[4], y[4], z[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int32_t p = pb + 32 * u + lane;
      if (p < p1) { x[u] = vx[p]; y[u] = vy[p]; z[u] = vz[p]; }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int32_t p = pb + 32 * u + lane;
      if (p < p1) {
        while (c < nc - 1 && p >= cs[c + 1]) ++c;
        const double* cf = coef[c];
        vx[p] = fma(cf[0], x[u], cf[1]);
        vy[p] = fma(cf[0], y[u], cf[2]);
        vz[p] = fma(cf[0], z[u], cf[3]);
      }
    }
  }
}

// Moments into mom (MATCH = false), or matching of the velocities to the
// pre-collision moments in mom (MATCH = true).
template <bool MATCH>
__global__ void __launch_bounds__(kCwWarps * 32, MATCH ? 3 : 4)
k_cells(int32_t n_cells, const int32_t* __restrict__ cs, double* vx, double* vy, double* vz, double* mom,
        int* status, unsigned* work) {
  __shared__ CwWarp sw[kCwWarps];
  CwWarp& W = sw[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31, sl = lane & (kSeg - 1), seg = lane / kSeg;
  for (;;) {
    int nclaim = 0;
    for (int q = 0; q < kCwClaims; ++q) {
      unsigned k0u = 0u;
      if (lane == 0) k0u = atomicAdd(work, (unsigned)kCwRun);
      k0u = __shfl_sync(0xffffffffu, k0u, 0);
      if (k0u >= (unsigned)n_cells) break;
      const int32_t k0 = (int32_t)k0u;
      const int nc = min(kCwRun, n_cells - k0);
      if (lane <= kCwRun) W.cs[q][lane] = cs[k0 + min(lane, nc)];
      if (lane == 0) W.k0[q] = k0;
      __syncwarp();
      for (int g = 0; g * 4 < nc; ++g) {
        const int ci = 4 * g + seg;
        const bool act = ci < nc;
        const int32_t a = act ? W.cs[q][ci] : 0, b = act ? W.cs[q][ci + 1] : 0;
        int E;
        const FixAcc f = cell_sums<kSeg>(vx, vy, vz, a, b, sl, &E);
        if (act && sl == 0) { W.acc[q * kCwRun + ci] = f; W.E[q * kCwRun + ci] = E; }
      }
      ++nclaim;
    }
    if (nclaim == 0) break;
    __syncwarp();
    {
      const int q = lane / kCwRun, ci = lane % kCwRun;
      const int32_t k = q < nclaim ? W.k0[q] + ci : n_cells;
      if (k < n_cells) {
        const int32_t n = W.cs[q][ci + 1] - W.cs[q][ci];
        const CellFix C = cellfix_from(W.E[lane], n, W.acc[lane]);
        double* mk = mom + 5 * (size_t)k;
        if (!MATCH) {
          for (int r = 0; r < 5; ++r) moment_store(C, n, r, mk, status);
        } else {
          double alpha, o[3];
          match_coeffs3(C, n, mk, &alpha, o);
          W.coef[lane][0] = alpha; W.coef[lane][1] = o[0]; W.coef[lane][2] = o[1]; W.coef[lane][3] = o[2];
        }
      }
    }
    __syncwarp();
    if (MATCH) {
      for (int q = 0; q < nclaim; ++q)
        apply_run(W.cs[q], min(kCwRun, n_cells - W.k0[q]), W.coef + q * kCwRun, vx, vy, vz);
    }
    __syncwarp();
    if (nclaim < kCwClaims) break;
  }
  // the last warp of the grid to finish resets the counters for the next
  // launch (the fences order every warp's last claim before the reset)
  if (lane == 0) {
    __threadfence();
    if (atomicAdd(work + 1, 1u) == gridDim.x * kCwWarps - 1) {
      __threadfence();
      work[0] = 0u;
      work[1] = 0u;
    }
  }
}

static int launch_cells(Ctx* c, bool match, int32_t n_cells, const int32_t* cs, double* vx, double* vy,
                        double* vz, double* mom, cudaStream_t s) {
  if (n_cells <= 0) return 0;
  const Shape sh = shape_or_default(c, match ? DSMC_TUNE_MOMENT_MATCH : DSMC_TUNE_MOMENTS);
  const int64_t runs = ((int64_t)n_cells + kCwRun - 1) / kCwRun;
  const unsigned g = grid_for(runs, kCwWarps * kCwClaims, sm_count(c) * sh.blocks_per_sm);
  if (match) k_cells<true><<<g, kCwWarps * 32, 0, s>>>(n_cells, cs, vx, vy, vz, mom, nullptr, work_ptr(c));
  else k_cells<false><<<g, kCwWarps * 32, 0, s>>>(n_cells, cs, vx, vy, vz, mom, status_ptr(c), work_ptr(c));
  count_launches(c, 1);
  return cudaGetLastError() == cudaSuccess ? 0 : DSMC_ERR_CUDA;
}

int launch_moments(Ctx* c, int32_t n_cells, const int32_t* cs, const double* vx, const double* vy,
                   const double* vz, double* mom, cudaStream_t s) {
  return launch_cells(c, false, n_cells, cs, (double*)vx, (double*)vy, (double*)vz, mom, s);
}

// ---------------------------------------------------------------- moment matching
// Sec. 2.5 (centred): v <- u_pre + alpha (v - u_post), alpha = sqrt(Th_pre/Th_post),
// applied as v <- alpha v + (u_pre - alpha u_post) (FP64); u_post and Th_post
// from the exact integer moments above (k_cells<true>).
int launch_moment_match(Ctx* c, int32_t n_cells, const int32_t* cs, const double* mom,
                        double* vx, double* vy, double* vz, cudaStream_t s) {
  return launch_cells(c, true, n_cells, cs, vx, vy, vz, (double*)mom, s);
}

}  // namespace dsmc

// ---------------------------------------------------------------- allocation-free sort
// A variant of the cell sort for callers that cannot allocate device memory.
// Its scratch (per-cell counters, the unsorted slot array, the scan's block
// sums and a spare status word) is one file-scope device array, so the call
// itself allocates nothing; every GPU that loads this library holds the
// array until the process exits.
#include <mutex>

namespace dsmc {

constexpr size_t kStaticCountsBytes = sizeof(int32_t) * (size_t)DSMC_STATIC_SORT_MAX_CELLS;
constexpr size_t kStaticSlotsBytes = sizeof(int32_t) * (size_t)DSMC_STATIC_SORT_MAX_N;
constexpr size_t kStaticScanBytes =
    sizeof(int32_t) * (size_t)((DSMC_STATIC_SORT_MAX_CELLS + kScanItems - 1) / kScanItems + 1);
constexpr size_t kStaticScanSlot = 512;  // block sums of the scan
constexpr size_t kStaticScratchBytes = kStaticCountsBytes + kStaticSlotsBytes + kStaticScanSlot + 256;

static __device__ __align__(256) unsigned char g_sort_scratch[kStaticScratchBytes];

namespace {
constexpr int kMaxDevices = 64;
struct StaticSortDevice {
  unsigned char* scratch = nullptr;  // device address of g_sort_scratch on this device
  int sms = 0;
};
StaticSortDevice g_static_dev[kMaxDevices];
std::mutex g_static_mu;
}  // namespace

// Once per device, with that device current: the device address of the
// scratch array (in host code its name only stands for the symbol) and the
// SM count used to size the grids.
static int static_sort_setup(int dev, StaticSortDevice** out) {
  std::lock_guard<std::mutex> lock(g_static_mu);
  StaticSortDevice& d = g_static_dev[dev];
  if (!d.scratch) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_sort_scratch) != cudaSuccess || !ptr) return DSMC_ERR_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
      return DSMC_ERR_CUDA;
    d.sms = sms;
    d.scratch = (unsigned char*)ptr;
  }
  *out = &d;
  return 0;
}

}  // namespace dsmc

extern "C" int dsmc_sort_cells_static(int32_t n, int32_t n_cells, const int32_t* cell_id,
                                      const double* vx, const double* vy, const double* vz,
                                      int32_t* perm, int32_t* cell_start, double* svx,
                                      double* svy, double* svz, int* status, void* stream) {
  using namespace dsmc;
  if (n < 0 || n_cells < 1 || !cell_start) return DSMC_ERR_ARG;
  if (n > DSMC_STATIC_SORT_MAX_N || n_cells > DSMC_STATIC_SORT_MAX_CELLS) return DSMC_ERR_UNSUPPORTED;
  if (n > 0 && !(cell_id && vx && vy && vz && perm && svx && svy && svz)) return DSMC_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DSMC_ERR_CUDA;
  StaticSortDevice* d = nullptr;
  if (int rc = static_sort_setup(dev, &d)) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  int32_t* counts = (int32_t*)d->scratch;
  int32_t* slots = (int32_t*)(d->scratch + kStaticCountsBytes);
  int32_t* scan = (int32_t*)(d->scratch + kStaticCountsBytes + kStaticSlotsBytes);
  int* st = status ? status : (int*)(d->scratch + kStaticCountsBytes + kStaticSlotsBytes + kStaticScanSlot);
  static_assert(kStaticScanBytes <= kStaticScanSlot, "scan block sums must fit their slot");
  static_assert(DSMC_STATIC_SORT_MAX_N <= (1 << (3 * kLgBits)), "three 8-bit passes order every slot value");
  // the counters must start at zero on every call (the array keeps the last call's contents)
  if (cudaMemsetAsync(counts, 0, sizeof(int32_t) * (size_t)n_cells, s) != cudaSuccess) return DSMC_ERR_CUDA;
  if (n > 0) k_hist<<<grid_for(n, 256, d->sms * 16), 256, 0, s>>>(cell_id, n, n_cells, counts, st);
  if (int rc = launch_scan(nullptr, counts, cell_start, n_cells, scan, s)) return rc;
  if (n > 0) {
    if (cudaMemsetAsync(counts, 0, sizeof(int32_t) * (size_t)n_cells, s) != cudaSuccess) return DSMC_ERR_CUDA;
    k_scatter<<<grid_for(n, 256, d->sms * 16), 256, 0, s>>>(cell_id, n, n_cells, cell_start, counts, slots);
    k_fix_gather<<<grid_for(n_cells, kFixWarps, d->sms * 4), kFixWarps * 32, 0, s>>>(n_cells, cell_start, slots,
                                                                                      perm);
    k_fix_large<<<grid_for(n_cells, 1, d->sms), kLgWarps * 32, 0, s>>>(n_cells, cell_start, slots, perm);
    k_gather<<<grid_for(n, 256, d->sms * 16), 256, 0, s>>>(n, cell_start, n_cells, perm, vx, vy, vz, svx,
                                                           svy, svz);
  }
  return cudaGetLastError() == cudaSuccess ? DSMC_OK : DSMC_ERR_CUDA;
}
