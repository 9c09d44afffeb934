// Internal device helpers and launcher declarations of the DSMC library.
// Target: sm_103a (GB300).  Everything here is the library's own code.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "dsmc.h"

#define DSMC_KB 1.380649e-23
#define DSMC_PI 3.14159265358979323846

namespace dsmc {

// Philox tags (counter word 3): 1 NTC rounding, 2 candidate, 3 isotropic
// direction, 4 Jager b/eps, 5 latent noise, 6 harvest.
enum : uint32_t { TAG_NTC = 1, TAG_CAND = 2, TAG_ISO = 3, TAG_JAGER = 4, TAG_NOISE = 5 };

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplies with the Weyl-sequence key schedule.
struct u32x4 { uint32_t x, y, z, w; };

__device__ __forceinline__ u32x4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  return {c0, c1, c2, c3};
}

// counter = (idx, cell, step_lo, tag | sub<<8 | step_hi<<16), key = seed
__device__ __forceinline__ u32x4 draw(uint64_t seed, uint32_t idx, uint32_t cell, uint64_t step,
                                      uint32_t tag, uint32_t sub = 0) {
  return philox(idx, cell, (uint32_t)step, tag | (sub << 8) | ((uint32_t)(step >> 32) << 16),
                (uint32_t)seed, (uint32_t)(seed >> 32));
}

// The same generator with its ten round keys formed once on the host (the
// Weyl sequence of the seed), so that inside a kernel they are launch
// constants: each round is then two multiplies and two three-way XORs with
// a constant operand, with no key arithmetic per draw.
struct PhiloxKey {
  uint32_t k0[10], k1[10];
};

inline PhiloxKey philox_key(uint64_t seed) {
  PhiloxKey K;
  uint32_t a = (uint32_t)seed, b = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    K.k0[r] = a; K.k1[r] = b;
    a += 0x9E3779B9u; b += 0xBB67AE85u;
  }
  return K;
}

__device__ __forceinline__ u32x4 draw_k(const PhiloxKey& K, uint32_t idx, uint32_t cell, uint64_t step,
                                        uint32_t tag, uint32_t sub = 0) {
  uint32_t c0 = idx, c1 = cell, c2 = (uint32_t)step, c3 = tag | (sub << 8) | ((uint32_t)(step >> 32) << 16);
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ K.k0[r], n2 = hi0 ^ c3 ^ K.k1[r];
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  return {c0, c1, c2, c3};
}

// 53-bit uniform in [0,1): exact in double
__device__ __forceinline__ double u53(uint32_t a, uint32_t b) {
  const uint64_t x = ((((uint64_t)a) << 32) | b) >> 11;
  return (double)x * (1.0 / 9007199254740992.0);
}

// the same uniform built on the integer pipe (no FP64 conversion): the
// 53-bit integer x = (a << 32 | b) >> 11 normalised into the fraction of a
// double, x 2^-53 exactly
__device__ __forceinline__ double u53_int(uint32_t a, uint32_t b) {
  const uint64_t x = ((((uint64_t)a) << 32) | b) >> 11;
  if (x == 0) return 0.0;
  const int lz = __clzll((long long)x) - 11;         // leading 1 moved to bit 52
  const uint64_t m = (x << lz) & 0xFFFFFFFFFFFFFull;
  const uint64_t e = (uint64_t)(1023 - 1 - lz);       // x 2^-53 = 1.m 2^(-1 - lz)
  return __longlong_as_double((long long)((e << 52) | m));
}

// the same uniform rounded to FP32 (within 2^-23 relative of u53(a, b);
// the low word matters below 2^-8)
__device__ __forceinline__ float u_f32(uint32_t a, uint32_t b) {
  return fmaf(__uint2float_rn(b >> 11), 0x1p-53f, __uint2float_rn(a) * 0x1p-32f);
}

// uniform integer in [0, n): high word of w*n
__device__ __forceinline__ uint32_t mulhi_n(uint32_t w, uint32_t n) { return __umulhi(w, n); }

__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------- status
// First error wins; later ones are dropped.
__device__ __forceinline__ void set_status(int* status, int code) {
  atomicCAS(status, 0, code);
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Device-wide barrier for a cooperative (co-resident) grid.  `bar[0]` counts
// arrivals, `bar[1]` is the generation.  Every wait is bounded: after
// `limit_ns` the block records DSMC_ERR_TIMEOUT, raises the abort flag
// bar[2] and returns false; callers then leave the kernel.
// bar[3] is a work cursor that the last block to arrive resets to 0 before
// releasing the others (every block has stopped claiming work by then).
__device__ __forceinline__ bool grid_barrier(unsigned* bar, int* status, uint64_t limit_ns) {
  __syncthreads();
  __shared__ int ok;
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* vgen = bar + 1;
    volatile unsigned* vabort = bar + 2;
    const unsigned gen = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u);
    if (arrived == gridDim.x - 1) {
      bar[0] = 0;
      bar[3] = 0;
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const uint64_t t0 = globaltimer_ns();
      while (*vgen == gen) {
        if (*vabort) { ok = 0; break; }
        if (globaltimer_ns() - t0 > limit_ns) {
          set_status(status, DSMC_ERR_TIMEOUT);
          atomicExch(bar + 2, 1u);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

constexpr uint64_t kBarrierLimitNs = 2000000000ull;  // 2 s

// FP64 -> FP32 with round-to-nearest-even on the integer pipe (GB300's FP64
// pipe, which also does the conversion instruction, is ~1/64 of FP32): keep
// the top 23 mantissa bits, round on the 29 dropped ones; results below the
// FP32 normal range become a signed zero.  Equal to the hardware conversion
// for every input of magnitude in [2^-126, FLT_MAX].
__device__ __forceinline__ float f64_to_f32(double v) {
  const uint32_t hi = (uint32_t)__double2hiint(v), lo = (uint32_t)__double2loint(v);
  const uint32_t sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu);
  const uint32_t m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  const uint32_t rest = lo & 0x1FFFFFFFu;
  uint32_t f = sign | ((uint32_t)(e - 896) << 23) | m;
  f += (rest > 0x10000000u) || (rest == 0x10000000u && (m & 1u));
  return __uint_as_float(e < 897 ? sign : f);
}

// FP32 -> FP64 (exact) on the integer pipe, from the IEEE-754 layouts: the
// exponent rebiased by 1023 - 127 = 896 and the 23-bit fraction placed at
// the top of the 52-bit one; subnormal inputs normalised first, zeros,
// infinities and NaNs kept.
__device__ __forceinline__ double f32_to_f64(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t sign = u & 0x80000000u;
  uint32_t e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
  uint32_t hi;
  if (e == 0xFFu) {
    hi = sign | 0x7FF00000u | (m >> 3);
  } else if (e == 0u && m == 0u) {
    hi = sign;
  } else {
    if (e == 0u) {   // subnormal: value 2^-126 m 2^-23, leading one moved to bit 23
      const uint32_t sh = (uint32_t)__clz(m) - 8u;
      m = (m << sh) & 0x7FFFFFu;
      e = 1u - sh;
    }
    hi = sign | ((e + 896u) << 20) | (m >> 3);
  }
  return __hiloint2double((int)hi, (int)(m << 29));
}

// ---------------------------------------------------------------- pair dependencies
// The collide kernels walk the pairs of a step in round-major order without
// grid-wide barriers.  Work units (a warp's 32 pairs, a 128-pair MLP tile)
// never span two rounds and are claimed in order from one global cursor; a
// pair starts once the previous pairs of its two particles are done.
// done[i] is the 1-based round of the last completed pair of particle i
// (zeroed before the launch); a pair's deps word holds the 1-based rounds of
// the previous pairs of its particles (low / high 16 bits, 0 = none), all
// below its own round.  A wait only ever points at pairs of units claimed
// earlier, so the earliest unfinished unit always has its inputs done: the
// scheme cannot deadlock, and every wait is bounded besides.

// Map claimed unit `unit` to its pair range [*p0, *p1) and round *r.  (r,
// base) is the caller's running position: round r starts at unit `base`;
// units are claimed in increasing order, so it only moves forward.  False
// once past the last round.
__device__ __forceinline__ bool unit_range(const int32_t* __restrict__ ro, int R, int usize, int& r,
                                           int64_t& base, int64_t unit, int32_t* p0, int32_t* p1) {
  while (r < R) {
    const int32_t b = ro[r], e = ro[r + 1];
    const int64_t nu = (e - b + usize - 1) / usize;
    if (unit < base + nu) {
      *p0 = b + (int32_t)((unit - base) * usize);
      *p1 = min(e, *p0 + usize);
      return true;
    }
    base += nu;
    ++r;
  }
  return false;
}

// Release / acquire at GPU scope (PTX memory model): a relaxed load of a
// stamp followed by fence.acq_rel is an acquire; fence.acq_rel followed by
// a relaxed store of the stamp is a release.  Lighter than fence.sc.
__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(unsigned* p, unsigned v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// Wait until the previous pairs of particles i and j are done (bounded; on
// timeout, or once another thread has aborted, records DSMC_ERR_TIMEOUT,
// raises the abort word and returns false).
__device__ __forceinline__ bool wait_deps(const unsigned* done, int32_t i, int32_t j, uint32_t dep,
                                          unsigned* abort_word, int* status,
                                          uint64_t limit_ns = kBarrierLimitNs) {
  const unsigned ni = dep & 0xFFFFu, nj = dep >> 16;
  if (ni == 0 && nj == 0) return true;
  if (ld_relaxed(done + i) >= ni && ld_relaxed(done + j) >= nj) { fence_acq_rel(); return true; }
  const uint64_t t0 = globaltimer_ns();
  unsigned sleep_ns = 32;   // doubling up to 1 us: a waiting lane costs few issue slots
  for (;;) {
    __nanosleep(sleep_ns);
    if (sleep_ns < 1024) sleep_ns <<= 1;
    if (ld_relaxed(done + i) >= ni && ld_relaxed(done + j) >= nj) { fence_acq_rel(); return true; }
    if (ld_relaxed(abort_word) || globaltimer_ns() - t0 > limit_ns) {
      set_status(status, DSMC_ERR_TIMEOUT);
      atomicExch(abort_word, 1u);
      return false;
    }
  }
}

// Publish that the pair of particles i and j (1-based round `round1`) is
// done: its velocity stores become visible before the stamps.
__device__ __forceinline__ void release_pair(unsigned* done, int32_t i, int32_t j, unsigned round1) {
  fence_acq_rel();
  st_relaxed(done + i, round1);
  st_relaxed(done + j, round1);
}

// ---------------------------------------------------------------- host side
struct Ctx;
int record(Ctx* c, int code, const char* msg);  // sets last error text, returns code
int* status_ptr(Ctx* c);
unsigned* barrier_ptr(Ctx* c);  // 4 words of device memory per barrier slot
// Two words of device memory for a work counter (next item, finished warps),
// zero between launches: the kernel that uses them leaves them zero.
unsigned* work_ptr(Ctx* c);
int sm_count(Ctx* c);
void count_launches(Ctx* c, int k);  // kernels launched by this context
// Device address the kernels read the step index from while a step graph is
// being captured (null otherwise: the step is then a kernel argument).
const uint64_t* graph_step_ptr(Ctx* c);

// launchers (return 0 or a DSMC_ERR_* code)
int launch_sort(Ctx* c, int32_t n, int32_t n_cells, const int32_t* cell_id, const double* vx,
                const double* vy, const double* vz, int32_t* perm, int32_t* cell_start,
                double* svx, double* svy, double* svz, void* ws, size_t ws_bytes,
                cudaStream_t s);
int launch_sort_keys(Ctx* c, int32_t n, int32_t n_cells, const int32_t* cell_id, int32_t* perm,
                     int32_t* cell_start, void* ws, size_t ws_bytes, cudaStream_t s);
size_t sort_ws(int32_t n, int32_t n_cells);
int launch_moments(Ctx* c, int32_t n_cells, const int32_t* cs, const double* vx,
                   const double* vy, const double* vz, double* mom, cudaStream_t s);
int launch_moment_match(Ctx* c, int32_t n_cells, const int32_t* cs, const double* mom,
                        double* vx, double* vy, double* vz, cudaStream_t s);
size_t select_ws(int32_t n, int32_t n_cells, int64_t capacity);
int launch_select(Ctx* c, const dsmc_gas_t& gas, int32_t n, int32_t n_cells, const int32_t* cs,
                  const double* vx, const double* vy, const double* vz, double* sgmax,
                  uint64_t step, int64_t capacity, int32_t* pairs, uint32_t* deps, int32_t* round_offsets,
                  dsmc_select_info_t* info, void* ws, size_t ws_bytes, int32_t order, cudaStream_t s);
int launch_sgmax_init(Ctx* c, const dsmc_gas_t& gas, int32_t n_cells, const double* T,
                      double factor, double* sgmax, cudaStream_t s);
// per-particle done stamps of the collide kernels
size_t collide_ws(int32_t n);
int launch_collide_vhs(Ctx* c, const dsmc_gas_t& gas, uint64_t step, int32_t n, const int32_t* pairs,
                       const uint32_t* deps, const int32_t* ro, const dsmc_select_info_t* info, double* vx,
                       double* vy, double* vz, void* ws, size_t ws_bytes, cudaStream_t s);
int launch_jager_chi(Ctx* c, const dsmc_gas_t& gas, const dsmc_potential_t& pot, int n_nodes,
                     int64_t n, const float* b, const float* g, float* chi, cudaStream_t s);
int launch_collide_jager(Ctx* c, const dsmc_gas_t& gas, const dsmc_potential_t& pot,
                         int n_nodes, uint64_t step, int32_t n, const int32_t* pairs, const uint32_t* deps,
                         const int32_t* ro, const dsmc_select_info_t* info, double* vx, double* vy,
                         double* vz, float* chi_out, void* ws, size_t ws_bytes, cudaStream_t s);
int launch_chi_table(Ctx* c, const dsmc_gas_t& gas, const dsmc_potential_t& pot, int n_nodes, int32_t nb,
                     int32_t nE, double lnE_min, double lnE_max, float* T, cudaStream_t s);
int launch_collide_table(Ctx* c, const dsmc_gas_t& gas, const dsmc_chi_table_t& tab, uint64_t step, int32_t n,
                         const int32_t* pairs, const uint32_t* deps, const int32_t* ro,
                         const dsmc_select_info_t* info, double* vx, double* vy, double* vz, float* chi_out,
                         void* ws, size_t ws_bytes, cudaStream_t s);
int occupancy_collide_table(int threads);
size_t transport_ws(int32_t n_T, int32_t x_panels);
size_t chi_mlp_packed_size();
int launch_chi_mlp_pack(Ctx* c, const uint16_t* w_bits, void* packed, cudaStream_t s);
int launch_chi_mlp_forward(Ctx* c, const void* packed, const float* bias, int64_t n, const float* x, float* y,
                           float* chi, cudaStream_t s);
int launch_chi_mlp_table(Ctx* c, const void* packed, const float* bias, int32_t nb, int32_t nE, float* table,
                         cudaStream_t s);
int launch_transport_q2(Ctx* c, const dsmc_potential_t& pot, int n_nodes, int32_t n_E, const double* E,
                        double bmax, int32_t b_panels, double* q2, cudaStream_t s);
int launch_transport_viscosity(Ctx* c, const dsmc_gas_t& gas, const dsmc_potential_t& pot, int n_nodes,
                               int32_t n_T, const double* T, double bmax, int32_t b_panels, int32_t x_panels,
                               double* omega22, double* mu, void* ws, size_t ws_bytes, cudaStream_t s);
int launch_harvest_jager(Ctx* c, const dsmc_gas_t& gas, const dsmc_potential_t& pot,
                         int n_nodes, int64_t n, const double* vi, const double* vj,
                         const double* b, const double* eps, double* vio, double* vjo,
                         cudaStream_t s);
int launch_collide_neural(Ctx* c, const dsmc_gas_t& gas, const dsmc_mlp_t& mlp,
                          const uint16_t* w, const float* bias, uint64_t step,
                          const double* mom, int32_t n, const int32_t* pairs, const uint32_t* deps,
                          const int32_t* ro, const dsmc_select_info_t* info, double* vx, double* vy,
                          double* vz, float* u_out, void* ws, size_t ws_bytes, cudaStream_t s);

int launch_mlp_forward(Ctx* c, const dsmc_mlp_t& mlp, const uint16_t* w, const float* bias,
                       int64_t n, const float* x, float* y, cudaStream_t s);
int launch_tc_selftest(Ctx* c, int N, int K, int layout, const uint16_t* A, const uint16_t* B, float* D,
                       cudaStream_t s);

// Launch shapes of the tunable kernels (DSMC_TUNE_*): threads per block and
// blocks per SM, {0, 0} while the built-in shape is in force.
struct Shape {
  int threads, blocks_per_sm;
};
Shape tune_shape(Ctx* c, int kernel);
// threads per block, blocks per SM and the block-size limit of the built-in shapes
struct ShapeInfo {
  int threads, blocks_per_sm, max_threads;
};
ShapeInfo shape_info(int kernel);
// the shape a launch uses: the tuned one, else the built-in one
inline Shape shape_or_default(Ctx* c, int kernel) {
  Shape s = tune_shape(c, kernel);
  if (s.threads <= 0) {
    const ShapeInfo d = shape_info(kernel);
    s = Shape{d.threads, d.blocks_per_sm};
  }
  return s;
}
// resident blocks per SM of the persistent collide kernels at a block size
int occupancy_collide_vhs(int threads);
int occupancy_collide_jager(int threads);
// the gather step of the cell sort alone (autotuning)
int launch_gather_one(Ctx* c, int32_t n, int32_t n_cells, const int32_t* cell_start, const int32_t* perm,
                      const double* v, double* sv, cudaStream_t s);
int launch_gather(Ctx* c, int32_t n, int32_t n_cells, const int32_t* cell_start, const int32_t* perm,
                  const double* vx, const double* vy, const double* vz, double* svx, double* svy,
                  double* svz, cudaStream_t s);
int launch_selftest_barrier(Ctx* c, uint64_t limit_ns, cudaStream_t s);
int64_t peak_ops_per_thread(int which, int32_t iters);
int launch_selftest_math(Ctx* c, int which, int64_t n, const double* x, double* y, cudaStream_t s);
int launch_peak(Ctx* c, int which, int32_t blocks, int32_t threads, int32_t iters, float* sink, cudaStream_t s);
int launch_selftest_deps(Ctx* c, uint64_t limit_ns, cudaStream_t s);
int launch_selftest_mbar(Ctx* c, uint64_t limit_ns, cudaStream_t s);

size_t train_ws(int sms);
int launch_train(Ctx* c, const dsmc_mlp_t& mlp, int mode, uint64_t seed, uint64_t t, int64_t n,
                 const float* theta, const double* vi, const double* vj, const double* T,
                 const double* ti, const double* tj, const double* gi, const double* gj, double* oi, double* oj,
                 float* grad, double* loss, void* ws, size_t ws_bytes, cudaStream_t s, float* act = nullptr);
size_t train_act_bytes(int64_t n);
int launch_adam(Ctx* c, int n_w, int n_b, const float* grad, float* master, float* m, float* v, uint16_t* w,
                float* bias, float lr, double b1, double b2, double eps, int64_t step, cudaStream_t s);

// the fused step (cell groups staged in shared memory), after the sort's keys
size_t fused_ws(int32_t n);
int launch_step_fused(Ctx* c, const dsmc_gas_t& gas, int path, const dsmc_chi_table_t* tab, uint64_t step,
                      int32_t n, int32_t n_cells, const int32_t* cs, const int32_t* perm, const double* vx,
                      const double* vy, const double* vz, double* svx, double* svy, double* svz, double* mom,
                      double* sgmax, int32_t* pairs, int64_t capacity, dsmc_select_info_t* info, void* ws,
                      size_t ws_bytes, cudaStream_t s);

// exclusive scan of int32 counts -> offsets[n+1] (offsets[n] = total)
size_t scan_ws(int64_t n);
int launch_scan(Ctx* c, const int32_t* in, int32_t* out, int64_t n, void* ws, cudaStream_t s);

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace dsmc
