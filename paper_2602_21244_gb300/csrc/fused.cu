// Fused collision step: after the cell sort's keys, one persistent kernel
// takes each cell's particles through the whole step -- gather, cell
// moments, NTC selection, rounds, pair updates, moment matching -- with the
// cell's velocities staged in shared memory once (Sec. 2.2-2.5 for the
// steps; the arithmetic is the unfused kernels', through the same device
// functions, so the two give bit-identical results).
//
// Cells are grouped by their first particle's sorted position: group g holds
// the cells that start in [g G, (g + 1) G) (G = kGroup particles), so every
// cell belongs to exactly one group and no group needs to know another's
// size (k_group_starts tabulates each group's first cell).  A CTA claims
// groups from a global cursor and cuts each into batches of consecutive
// cells that fit in shared memory (kFCap particles, kFCand candidates,
// kFCells cells).  Per batch:
//   P0  per cell N and the NTC candidate count M; the batch's extent
//   P1  gather the batch's velocities (perm) into shared memory, FP64 and an
//       FP32 copy for the screen
//   P2  exact integer cell moments, one warp per cell; their FP64 values
//       (written out: the matching targets), one thread per cell; the
//       screen constants
//   P3  every candidate of the batch evaluated in parallel (one thread per
//       candidate): particles, screened exact accept decision, (sigma g)_max
//   P4  rounds in candidate order, one warp per cell, 32 accepted
//       candidates at a time (batch_rounds)
//   P5  the accepted pairs bucketed by round
//   P6  the pair updates round by round (pairs of a round are disjoint)
//   P7  moment matching: post moments per warp, coefficients per thread,
//       the update per warp
//   P8  the sorted, post-collision velocities written out
// A single cell too large for shared memory runs the same phases on
// global-memory scratch (FP32 copies, masks and rounds in the workspace,
// its candidates in the caller's pair buffer).
//
// HBM traffic per particle: its index (4 B), its three input components
// (24 B, gathered) and three output components (24 B), against the unfused
// step's re-reads of the sorted arrays in every phase.  On GB300 the
// unfused step is nevertheless the faster one: its phases run far below
// the HBM roof (latency- and FP64-bound), while here each batch walks its
// phases and rounds behind block barriers with few batches per SM, and the
// round-synchronous pair updates leave GB300's FP64 warps partly filled.
#include "internal.cuh"
#include "moments.cuh"
#include "pair.cuh"
#include "select.cuh"

namespace dsmc {

constexpr int kFThreads = 256;
constexpr int kFWarps = kFThreads / 32;
constexpr int32_t kGroup = 512;   // particle stride of the cell groups
constexpr int kFCap = 1024;       // particles of a batch in shared memory
constexpr int kFCand = 3072;      // candidates of a batch
constexpr int kFCells = 128;      // cells of a batch
constexpr uint16_t kRejected = 0xFFFF;

struct FusedShared {
  double vx[kFCap], vy[kFCap], vz[kFCap];
  union {
    float f[3 * kFCap];            // P1-P3: FP32 copies for the screen
    struct {
      uint32_t msk[kFCap];         // P4: lane masks of batch_rounds
      uint16_t order[kFCand];      // P5-P6: candidates in round-major order
    } r;
  } u;
  uint16_t last[kFCap];            // P4: 1-based round of each particle's last pair
  uint32_t pij[kFCand];            // batch-local particles i | j << 16
  uint16_t pk[kFCand];             // batch-local cell
  uint16_t pround[kFCand];         // 0-based round, kRejected if not accepted
  int32_t cN[kFCells], cM[kFCells];
  int32_t cstart[kFCells + 1], cmofs[kFCells + 1];  // batch-local first particle / candidate
  double csg[kFCells];             // (sigma g)_max at the start of the step
  long long cbest[kFCells];        // new (sigma g)_max, as int64 bit patterns
  float cdg[kFCells], csg32[kFCells];
  int32_t rcount[DSMC_MAX_ROUNDS + 1];  // per round: count, then start, then end
  int32_t scan_tmp[2 * kFWarps];
  int32_t group, k0, k1, skip, rmax, npairs;
  long long gofs;
};

struct FusedArgs {
  SelArgs sel;                     // seed, step, NTC and cross-section constants, sgmax, status
  TableLook look;
  const int32_t* cs;
  const int32_t* perm;
  const double *vx, *vy, *vz;      // unsorted input
  double *svx, *svy, *svz;         // sorted post-collision output
  double* mom;
  dsmc_select_info_t* info;
  float* gf;                       // 3 n: FP32 copies of a large cell
  uint32_t* gmsk;                  // n
  uint16_t* glast;                 // n
  uint32_t* gcand;                 // candidate scratch of large cells (12 B per candidate)
  long long gcap;                  // its capacity in candidates
  const int32_t* gstart;           // first cell of each group ([n_groups] = n_cells)
  unsigned* bar;                   // [0] scratch cursor, [3] group cursor
  int* status;
  int32_t n, n_cells, n_groups;
};

// Arrays of one batch: shared memory, or global scratch for a large cell.
template <class OrderT>
struct Mem {
  double *vx, *vy, *vz;
  float *fx, *fy, *fz;
  uint32_t* msk;
  uint16_t* last;
  uint32_t* pij;
  uint16_t* pk;
  uint16_t* pround;
  OrderT* order;
};

// First cell of every group: gstart[g] = the first k in [0, n_cells) with
// cs[k] >= g G (n_cells if none), gstart[n_groups] = n_cells.  Cell k is the
// first cell of the groups g with cs[k-1] < g G <= cs[k] (cs[-1] = -1).
__global__ void k_group_starts(const int32_t* __restrict__ cs, int32_t n_cells, int32_t n_groups,
                               int32_t* __restrict__ gstart) {
  for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k <= n_cells; k += gridDim.x * blockDim.x) {
    if (k == n_cells) {
      // groups past the last cell start: empty
      const int32_t lo = n_cells > 0 ? cs[n_cells - 1] / kGroup + 1 : 0;
      for (int32_t g = lo; g <= n_groups; ++g) gstart[g] = n_cells;
      continue;
    }
    const int32_t g0 = k > 0 ? cs[k - 1] / kGroup + 1 : 0, g1 = cs[k] / kGroup;
    for (int32_t g = g0; g <= g1 && g < n_groups; ++g) gstart[g] = k;
  }
}

// Inclusive sums of (x, y) over threads 0..127 of the block (called by all
// threads; the others pass zeros).
__device__ __forceinline__ void scan128x2(int& x, int& y, int32_t* tmp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int xv = __shfl_up_sync(0xffffffffu, x, o), yv = __shfl_up_sync(0xffffffffu, y, o);
    if (lane >= o) { x += xv; y += yv; }
  }
  if (lane == 31 && warp < 4) { tmp[warp] = x; tmp[kFWarps + warp] = y; }
  __syncthreads();
  if (warp < 4) {
    for (int w = 0; w < warp; ++w) { x += tmp[w]; y += tmp[kFWarps + w]; }
  }
  __syncthreads();
}

// In place: a[0..R) -> exclusive prefix sums (R <= DSMC_MAX_ROUNDS).
constexpr int kScanPer = (DSMC_MAX_ROUNDS + kFThreads - 1) / kFThreads;

__device__ __forceinline__ void scan_excl(int32_t* a, int R, int32_t* tmp) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  int v[kScanPer], s = 0;
#pragma unroll
  for (int q = 0; q < kScanPer; ++q) {
    const int r = kScanPer * t + q;
    v[q] = r < R ? a[r] : 0;
    s += v[q];
  }
  int incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) tmp[warp] = incl;
  __syncthreads();
  int base = incl - s;
  for (int w = 0; w < warp; ++w) base += tmp[w];
#pragma unroll
  for (int q = 0; q < kScanPer; ++q) {
    const int r = kScanPer * t + q;
    if (r < R) a[r] = base;
    base += v[q];
  }
  __syncthreads();
}

// P1-P8 for the batch of cells [kb, kb + c) (particles [b0, b0 + P),
// candidates [0, Mb)); all threads of the block.
template <int PATH, class OrderT>
__device__ __forceinline__ void run_batch(const FusedArgs& a, FusedShared& S, const Mem<OrderT>& mem, int32_t kb, int c,
                          int32_t b0, int32_t P, int32_t Mb, bool in_smem) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool skip = S.skip != 0;
  // P1: gather (kFCap / kFThreads particles per thread, loads issued together)
  constexpr int kPer = kFCap / kFThreads;
  for (int32_t t0 = 0; t0 < P; t0 += kFCap) {
    int32_t idx[kPer];
    double x[kPer], y[kPer], z[kPer];
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int32_t t = t0 + tid + u * kFThreads;
      idx[u] = t < P ? __ldg(a.perm + b0 + t) : -1;
    }
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      if (idx[u] >= 0) { x[u] = __ldg(a.vx + idx[u]); y[u] = __ldg(a.vy + idx[u]); z[u] = __ldg(a.vz + idx[u]); }
    }
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int32_t t = t0 + tid + u * kFThreads;
      if (idx[u] >= 0) {
        mem.vx[t] = x[u]; mem.vy[t] = y[u]; mem.vz[t] = z[u];
        mem.fx[t] = f64_to_f32(x[u]); mem.fy[t] = f64_to_f32(y[u]); mem.fz[t] = f64_to_f32(z[u]);
        mem.last[t] = 0;
      }
    }
  }
  for (int r = tid; r <= DSMC_MAX_ROUNDS; r += kFThreads) S.rcount[r] = 0;
  if (tid == 0) { S.rmax = 0; S.npairs = 0; }
  __syncthreads();
  // P2: exact integer moments, one warp per cell (32 lanes over its
  // particles), and the screen constants; then the FP64 moments, one thread
  // per cell (GB300's FP64 pipe charges a whole warp instruction however
  // few lanes are active: one cell per lane, not one per warp)
  CellFix* cfix = reinterpret_cast<CellFix*>(S.pij);   // the candidate arrays are not yet in use
  for (int ci = warp; ci < c; ci += kFWarps) {
    const int32_t ls = S.cstart[ci], le = S.cstart[ci + 1];
    const CellFix C = cell_fix<32>(mem.vx, mem.vy, mem.vz, ls, le, lane);
    float vmax = 0.f;
    for (int32_t i = ls + lane; i < le; i += 32)
      vmax = fmaxf(vmax, fmaxf(fabsf(mem.fx[i]), fmaxf(fabsf(mem.fy[i]), fabsf(mem.fz[i]))));
    // non-negative floats: their bit patterns order as their values
    const float vm = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(vmax)));
    if (lane == 0) {
      cfix[ci] = C;
      // each FP32 velocity carries <= |v| 2^-24 rounding; g over three differences
      S.cdg[ci] = 4.0f * vm * 5.9604645e-8f;
      S.csg32[ci] = f64_to_f32(S.csg[ci]);
      S.cbest[ci] = __double_as_longlong(S.csg[ci]);
    }
  }
  __syncthreads();
  for (int ci = tid; ci < c; ci += kFThreads) {
    const CellFix C = cfix[ci];
    const int32_t n = S.cstart[ci + 1] - S.cstart[ci];
    double* mk = a.mom + 5 * (size_t)(kb + ci);
#pragma unroll
    for (int sl = 0; sl < 5; ++sl) moment_store(C, n, sl, mk, a.status);
  }
  __syncthreads();
  // P3: candidates, one thread each
  for (int32_t s = skip ? Mb : tid; s < Mb; s += kFThreads) {
    int lo = 0, hi = c - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (S.cmofs[mid] <= s) lo = mid;
      else hi = mid - 1;
    }
    const int ci = lo;
    const int32_t ls = S.cstart[ci];
    CellView cv;
    cv.x = mem.fx + ls; cv.y = mem.fy + ls; cv.z = mem.fz + ls;
    cv.v4 = nullptr;
    cv.dg = S.cdg[ci];
    cv.sgmax32 = S.csg32[ci];
    cv.inv_sgmax32 = 1.f / cv.sgmax32;
    cv.thr_raise = cv.sgmax32 * (1.f - 3e-4f);
    int32_t i, j;
    double sg = -1.0;
    const bool ok = candidate(a.sel, cv, CellRef{mem.vx, mem.vy, mem.vz, ls}, kb + ci, S.cN[ci], s - S.cmofs[ci],
                              S.csg[ci], &i, &j, &sg);
    mem.pij[s] = (uint32_t)(ls + i) | ((uint32_t)(ls + j) << 16);
    mem.pk[s] = (uint16_t)ci;
    mem.pround[s] = ok ? 0 : kRejected;
    if (sg >= 0.0) atomicMax(&S.cbest[ci], __double_as_longlong(sg));
  }
  __syncthreads();
  // P4: rounds in candidate order, one warp per cell, 32 accepted
  // candidates at a time (compacted through a per-warp queue); the new
  // (sigma g)_max
  uint32_t* queue = reinterpret_cast<uint32_t*>(S.u.r.order) + warp * 64;   // order is written in P5
  for (int ci = warp; ci < c; ci += kFWarps) {
    const int32_t ls = S.cstart[ci], le = S.cstart[ci + 1];
    for (int32_t i = ls + lane; i < le; i += 32) mem.msk[i] = 0u;
    __syncwarp();
    const int32_t s0 = skip ? 0 : S.cmofs[ci], s1 = skip ? 0 : S.cmofs[ci + 1];
    int cnt = 0, rm = -1, pending = 0;
    for (int32_t b = s0; b < s1 || pending > 0; b += 32) {
      const int32_t s = b + lane;
      const bool acc = s < s1 && mem.pround[s] == 0;
      const unsigned am = __ballot_sync(0xffffffffu, acc);
      if (acc) queue[pending + __popc(am & ((1u << lane) - 1u))] = (uint32_t)s;
      pending += __popc(am);
      __syncwarp();
      // a full batch, or the last one
      if (pending >= 32 || (b + 32 >= s1 && pending > 0)) {
        const bool act = lane < pending;
        const uint32_t q = act ? queue[lane] : 0u;
        const uint32_t ij = act ? mem.pij[q] : 0u;
        int Li, Lj;
        const int r = batch_rounds(act, ij & 0xFFFFu, ij >> 16, mem.msk, mem.last, a.status, &Li, &Lj);
        if (act) {
          mem.pround[q] = (uint16_t)r;
          ++cnt;
          rm = r > rm ? r : rm;
          atomicAdd(&S.rcount[r], 1);
        }
        const int rest = pending > 32 ? pending - 32 : 0;
        const uint32_t carry = lane < rest ? queue[32 + lane] : 0u;
        __syncwarp();
        if (lane < rest) queue[lane] = carry;
        pending = rest;
        __syncwarp();
      }
    }
    cnt = warp_sum_i(cnt);
    rm = __reduce_max_sync(0xffffffffu, rm);
    if (lane == 0) {
      if (cnt) atomicAdd(&S.npairs, cnt);
      if (rm >= 0) atomicMax(&S.rmax, rm + 1);
      if (!skip) a.sel.sgmax[kb + ci] = __longlong_as_double(S.cbest[ci]);
    }
  }
  __syncthreads();
  // P5: bucket the accepted candidates by round
  const int R = S.rmax;
  scan_excl(S.rcount, R, S.scan_tmp);
  for (int32_t s = tid; s < Mb && R > 0; s += kFThreads) {
    const uint16_t r = mem.pround[s];
    if (r != kRejected) mem.order[atomicAdd(&S.rcount[r], 1)] = (OrderT)s;
  }
  __syncthreads();
  // P6: pair updates, round by round (rcount[r] now holds the end of round r)
  for (int r = 0; r < R; ++r) {
    const int32_t q0 = r ? S.rcount[r - 1] : 0, q1 = S.rcount[r];
    for (int32_t q = q0 + tid; q < q1; q += kFThreads) {
      const uint32_t s = (uint32_t)mem.order[q];
      const uint32_t ij = mem.pij[s];
      const uint32_t i = ij & 0xFFFFu, j = ij >> 16;
      const int ci = mem.pk[s];
      const uint32_t m = s - (uint32_t)S.cmofs[ci], k = (uint32_t)(kb + ci);
      double v[6] = {mem.vx[i], mem.vy[i], mem.vz[i], mem.vx[j], mem.vy[j], mem.vz[j]};
      if (PATH == DSMC_PATH_TABLE) table_pair(a.look, a.sel.seed, a.sel.step, m, k, v);
      else vhs_pair(a.sel.seed, a.sel.step, m, k, v);
      mem.vx[i] = v[0]; mem.vy[i] = v[1]; mem.vz[i] = v[2];
      mem.vx[j] = v[3]; mem.vy[j] = v[4]; mem.vz[j] = v[5];
    }
    __syncthreads();
  }
  // P7: moment matching: integer post moments one warp per cell, the
  // coefficients one thread per cell, the update one warp per cell
  for (int ci = warp; ci < c; ci += kFWarps) {
    const CellFix C = cell_fix<32>(mem.vx, mem.vy, mem.vz, S.cstart[ci], S.cstart[ci + 1], lane);
    if (lane == 0) cfix[ci] = C;
  }
  __syncthreads();
  double* coef = reinterpret_cast<double*>(S.pk);   // alpha, ox, oy, oz per cell (pk, pround are dead)
  for (int ci = tid; ci < c; ci += kFThreads) {
    double alpha, o[3];
    match_coeffs3(cfix[ci], S.cstart[ci + 1] - S.cstart[ci], a.mom + 5 * (size_t)(kb + ci), &alpha, o);
    coef[4 * ci] = alpha; coef[4 * ci + 1] = o[0]; coef[4 * ci + 2] = o[1]; coef[4 * ci + 3] = o[2];
  }
  __syncthreads();
  for (int ci = warp; ci < c; ci += kFWarps) {
    const double alpha = coef[4 * ci], ox = coef[4 * ci + 1], oy = coef[4 * ci + 2], oz = coef[4 * ci + 3];
    for (int32_t i = S.cstart[ci] + lane; i < S.cstart[ci + 1]; i += 32) {
      mem.vx[i] = fma(alpha, mem.vx[i], ox);
      mem.vy[i] = fma(alpha, mem.vy[i], oy);
      mem.vz[i] = fma(alpha, mem.vz[i], oz);
    }
  }
  __syncthreads();
  // P8: write out
  if (in_smem) {
    for (int32_t t = tid; t < P; t += kFThreads) {
      a.svx[b0 + t] = mem.vx[t]; a.svy[b0 + t] = mem.vy[t]; a.svz[b0 + t] = mem.vz[t];
    }
  }
  if (tid == 0) {
    if (S.npairs) atomicAdd((unsigned long long*)&a.info->n_pairs, (unsigned long long)S.npairs);
    if (Mb) atomicAdd((unsigned long long*)&a.info->n_candidates, (unsigned long long)Mb);
    if (R) atomicMax(&a.info->n_rounds, R);
  }
  __syncthreads();
}

template <int PATH>
__global__ void __launch_bounds__(kFThreads, 3) k_step_fused(FusedArgs a) {
  extern __shared__ __align__(16) char smem_raw[];
  FusedShared& S = *reinterpret_cast<FusedShared*>(smem_raw);
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) {
      const int32_t g = (int32_t)atomicAdd(a.bar + 3, 1u);
      S.group = g;
      if (g < a.n_groups) {
        S.k0 = a.gstart[g];
        S.k1 = a.gstart[g + 1];
      }
    }
    __syncthreads();
    if (S.group >= a.n_groups) break;
    const int32_t k1 = S.k1;
    int32_t kb = S.k0;
    while (kb < k1) {
      // P0: the window's cells, N and M, and the longest prefix that fits
      const int w = min(kFCells, k1 - kb);
      int nx = 0, mx = 0;
      if (tid < w) {
        const int32_t k = kb + tid;
        const int32_t N = a.cs[k + 1] - a.cs[k];
        int bad = 0;
        const int32_t M = N < 2 ? 0 : ntc_count(a.sel, k, N, &bad);
        if (bad) set_status(a.status, DSMC_ERR_CAPACITY);
        S.cN[tid] = N; S.cM[tid] = M; S.csg[tid] = a.sel.sgmax[k];
        nx = min(N, kFCap + 1);
        mx = min(M, kFCand + 1);
      }
      scan128x2(nx, mx, S.scan_tmp);
      const bool fits = tid < w && nx <= kFCap && mx <= kFCand;
      int c = __syncthreads_count(fits);
      const bool big = c == 0;
      if (big) c = 1;
      if (tid < c) {
        S.cstart[tid] = a.cs[kb + tid] - a.cs[kb];
        S.cmofs[tid] = big ? 0 : mx - min(S.cM[tid], kFCand + 1);
      }
      if (tid == 0) {
        S.cstart[c] = a.cs[kb + c] - a.cs[kb];
        if (big) S.cmofs[1] = S.cM[0];
        S.skip = 0;
        if (big) {
          // a cell that alone exceeds the shared-memory batch: its candidates
          // take scratch in the caller's pair buffer
          const long long M = S.cM[0];
          if (S.cN[0] > 65536) {
            set_status(a.status, DSMC_ERR_UNSUPPORTED);
            S.skip = 1;
          } else {
            const unsigned long long off = atomicAdd((unsigned long long*)(a.bar), (unsigned long long)M);
            if ((long long)off + M > a.gcap) {
              set_status(a.status, DSMC_ERR_CAPACITY);
              S.skip = 1;
            }
            S.gofs = (long long)off;
          }
        }
      }
      if (tid == c - 1 && !big) S.cmofs[c] = mx;
      __syncthreads();
      const int32_t b0 = a.cs[kb], P = S.cstart[c];
      const int32_t Mb = S.cmofs[c];
      if (!big) {
        Mem<uint16_t> mem{S.vx, S.vy, S.vz, S.u.f, S.u.f + kFCap, S.u.f + 2 * kFCap, S.u.r.msk, S.last,
                          S.pij, S.pk, S.pround, S.u.r.order};
        run_batch<PATH, uint16_t>(a, S, mem, kb, c, b0, P, Mb, true);
      } else {
        const long long cap = a.gcap, off = S.skip ? 0 : S.gofs;
        uint32_t* pij = a.gcand + off;
        uint16_t* pk = (uint16_t*)(a.gcand + cap) + off;
        uint16_t* pr = (uint16_t*)(a.gcand + cap) + cap + off;
        uint32_t* ord = a.gcand + 2 * cap + off;
        Mem<uint32_t> mem{a.svx + b0, a.svy + b0, a.svz + b0, a.gf + b0, a.gf + a.n + b0, a.gf + 2 * (size_t)a.n + b0,
                          a.gmsk + b0, a.glast + b0, pij, pk, pr, ord};
        run_batch<PATH, uint32_t>(a, S, mem, kb, 1, b0, P, S.skip ? 0 : Mb, false);
      }
      kb += c;
    }
    __syncthreads();   // every thread is past S.group before thread 0 claims the next group
  }
}

static_assert(sizeof(FusedShared) <= 74 * 1024, "three CTAs per SM");
static_assert(kFCells <= 128 && kFThreads >= 128, "P0 scans 128 cells");
static_assert(sizeof(CellFix) * kFCells <= sizeof(uint32_t) * kFCand, "per-cell moments alias pij");
static_assert(sizeof(double) * 4 * kFCells <= sizeof(uint16_t) * 2 * kFCand, "coefficients alias pk, pround");
static_assert(sizeof(uint32_t) * 64 * kFWarps <= sizeof(uint16_t) * kFCand, "P4 queues alias order");

size_t fused_ws(int32_t n) {
  const size_t nn = (size_t)(n > 0 ? n : 1);
  return align256(12 * nn) + align256(4 * nn) + align256(2 * nn) + align256(4 * ((size_t)(n / kGroup) + 2));
}

int launch_step_fused(Ctx* c, const dsmc_gas_t& gas, int path, const dsmc_chi_table_t* tab, uint64_t step,
                      int32_t n, int32_t n_cells, const int32_t* cs, const int32_t* perm, const double* vx,
                      const double* vy, const double* vz, double* svx, double* svy, double* svz, double* mom,
                      double* sgmax, int32_t* pairs, int64_t capacity, dsmc_select_info_t* info, void* ws,
                      size_t ws_bytes, cudaStream_t s) {
  if (path != DSMC_PATH_VHS && path != DSMC_PATH_TABLE)
    return record(c, DSMC_ERR_UNSUPPORTED, "step_fused: VHS and look-up paths only");
  if (ws_bytes < fused_ws(n)) return record(c, DSMC_ERR_ARG, "step_fused: workspace too small");
  FusedArgs a;
  a.sel = SelArgs{};
  a.sel.sgmax = sgmax; a.sel.status = status_ptr(c); a.sel.n_cells = n_cells;
  a.sel.seed = gas.seed; a.sel.key = philox_key(gas.seed); a.sel.step = step; a.sel.step_dev = nullptr;   // not captured in the step graph
  a.sel.fn = gas.fn_over_vc; a.sel.dt = gas.dt;
  sel_model(a.sel, gas);
  a.look = path == DSMC_PATH_TABLE ? table_look(gas, *tab) : TableLook{};
  a.cs = cs; a.perm = perm; a.vx = vx; a.vy = vy; a.vz = vz; a.svx = svx; a.svy = svy; a.svz = svz;
  a.mom = mom; a.info = info;
  const size_t nn = (size_t)(n > 0 ? n : 1);
  char* p = (char*)ws;
  a.gf = (float*)p; p += align256(12 * nn);
  a.gmsk = (uint32_t*)p; p += align256(4 * nn);
  a.glast = (uint16_t*)p; p += align256(2 * nn);
  int32_t* gstart = (int32_t*)p;
  a.gstart = gstart;
  a.gcand = (uint32_t*)pairs;
  a.gcap = (long long)capacity;   // 12 of the 16 bytes of each pair slot
  a.bar = barrier_ptr(c); a.status = status_ptr(c);
  a.n = n; a.n_cells = n_cells; a.n_groups = n / kGroup + 1;
  const void* k = path == DSMC_PATH_TABLE ? (const void*)k_step_fused<DSMC_PATH_TABLE>
                                          : (const void*)k_step_fused<DSMC_PATH_VHS>;
  const int smem = (int)sizeof(FusedShared);
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
    return record(c, DSMC_ERR_CUDA, "step_fused: shared-memory attribute");
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kFThreads, smem) != cudaSuccess || per_sm < 1)
    return record(c, DSMC_ERR_CUDA, "step_fused: occupancy query failed");
  int64_t blocks = (int64_t)sm_count(c) * per_sm;
  if (blocks > a.n_groups) blocks = a.n_groups;
  if (cudaMemsetAsync(a.bar, 0, 4 * sizeof(unsigned), s) != cudaSuccess ||
      cudaMemsetAsync(info, 0, sizeof(dsmc_select_info_t), s) != cudaSuccess)
    return DSMC_ERR_CUDA;
  const int64_t gb = (n_cells + 1 + 255) / 256;
  k_group_starts<<<(unsigned)(gb < 4096 ? gb : 4096), 256, 0, s>>>(cs, n_cells, a.n_groups, gstart);
  if (path == DSMC_PATH_TABLE) k_step_fused<DSMC_PATH_TABLE><<<(unsigned)blocks, kFThreads, smem, s>>>(a);
  else k_step_fused<DSMC_PATH_VHS><<<(unsigned)blocks, kFThreads, smem, s>>>(a);
  count_launches(c, 2);
  return cudaGetLastError() == cudaSuccess ? 0 : record(c, DSMC_ERR_CUDA, "step_fused: launch failed");
}

}  // namespace dsmc
