// VHS isotropic scatter with the centre-of-mass update (Sec. 2.1, 2.3).
//
// One persistent launch walks the pairs of the step in round-major order:
// each warp claims 32 pairs of one round at a time from a global cursor and
// each lane waits (bounded) until the previous pairs of its two particles
// are done, then updates its pair and stamps both particles done.  The
// pairs of a round are disjoint, so no two lanes of a unit touch the same
// particle.  Velocities are read and written through L2 (ld/st .cg).
#include "internal.cuh"
#include "pair.cuh"

namespace dsmc {

struct VhsArgs {
  uint64_t seed, step;
  const uint64_t* step_dev;
  const int4* pairs;
  const uint32_t* deps;
  const int32_t* ro;
  const dsmc_select_info_t* info;
  double *vx, *vy, *vz;
  unsigned* done;
  unsigned* bar;   // [2] abort word, [3] unit cursor
  int* status;
};

__global__ void __launch_bounds__(256) k_collide_vhs(VhsArgs a) {
  if (a.step_dev) a.step = *a.step_dev;
  const int R = a.info->n_rounds;
  const int lane = threadIdx.x & 31;
  int r = 0;
  int64_t base = 0;
  // the next unit claimed and its pair records loading while the current
  // one updates (as in k_collide_table)
  auto claim = [&](int32_t* u0, int32_t* u1, int* ur) {
    unsigned unit = 0;
    if (lane == 0) unit = atomicAdd(a.bar + 3, 1u);
    unit = __shfl_sync(0xffffffffu, unit, 0);
    const bool got = unit_range(a.ro, R, 32, r, base, unit, u0, u1);
    *ur = r;
    return got;
  };
  int32_t p0 = 0, p1 = 0;
  int rc = 0;
  bool have = claim(&p0, &p1, &rc);
  int4 q = make_int4(0, 0, 0, 0);
  uint32_t dep = 0u;
  if (have && p0 + lane < p1) { q = a.pairs[p0 + lane]; dep = a.deps[p0 + lane]; }
  while (have) {
    int32_t n0 = 0, n1 = 0;
    int rn = 0;
    const bool next = claim(&n0, &n1, &rn);
    int4 qn = make_int4(0, 0, 0, 0);
    uint32_t depn = 0u;
    if (next && n0 + lane < n1) { qn = a.pairs[n0 + lane]; depn = a.deps[n0 + lane]; }
    const bool valid = p0 + lane < p1;
    bool ok = true;
    if (valid) ok = wait_deps(a.done, q.x, q.y, dep, a.bar + 2, a.status);
    const bool live = valid && ok;
    double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (live) {
      v[0] = __ldcg(a.vx + q.x); v[1] = __ldcg(a.vy + q.x); v[2] = __ldcg(a.vz + q.x);
      v[3] = __ldcg(a.vx + q.y); v[4] = __ldcg(a.vy + q.y); v[5] = __ldcg(a.vz + q.y);
    }
    // the lanes leave their dependency waits at different times: every lane
    // runs the pair update together after the warp reconverges (a lane
    // without a pair on zero velocities, its result not stored), since
    // GB300's FP64 pipe costs a warp instruction however few lanes are active
    __syncwarp();
    vhs_pair(a.seed, a.step, (uint32_t)q.w, (uint32_t)q.z, v);
    if (live) {
      __stcg(a.vx + q.x, v[0]); __stcg(a.vy + q.x, v[1]); __stcg(a.vz + q.x, v[2]);
      __stcg(a.vx + q.y, v[3]); __stcg(a.vy + q.y, v[4]); __stcg(a.vz + q.y, v[5]);
      release_pair(a.done, q.x, q.y, (unsigned)(rc + 1));
    }
    if (!__all_sync(0xffffffffu, ok)) break;
    have = next; p0 = n0; p1 = n1; rc = rn; q = qn; dep = depn;
  }
}


// resident blocks per SM of the VHS collide at a block size (0 on failure)
int occupancy_collide_vhs(int threads) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k_collide_vhs, threads, 0) != cudaSuccess)
    return 0;
  return per_sm;
}

size_t collide_ws(int32_t n) { return align256(sizeof(unsigned) * (size_t)(n > 0 ? n : 1)); }

int launch_collide_vhs(Ctx* c, const dsmc_gas_t& gas, uint64_t step, int32_t n, const int32_t* pairs,
                       const uint32_t* deps, const int32_t* ro, const dsmc_select_info_t* info, double* vx,
                       double* vy, double* vz, void* ws, size_t ws_bytes, cudaStream_t s) {
  if (ws_bytes < collide_ws(n)) return record(c, DSMC_ERR_ARG, "collide_vhs: workspace too small");
  const Shape sh = shape_or_default(c, DSMC_TUNE_COLLIDE_VHS);
  const int occ = occupancy_collide_vhs(sh.threads);
  if (occ < 1) return record(c, DSMC_ERR_CUDA, "collide_vhs: occupancy query failed");
  const int blocks = sm_count(c) * (sh.blocks_per_sm > 0 && sh.blocks_per_sm < occ ? sh.blocks_per_sm : occ);
  VhsArgs a{gas.seed, step, graph_step_ptr(c), (const int4*)pairs, deps, ro, info, vx, vy, vz,
            (unsigned*)ws, barrier_ptr(c), status_ptr(c)};
  if (cudaMemsetAsync(a.bar, 0, 4 * sizeof(unsigned), s) != cudaSuccess ||
      cudaMemsetAsync(a.done, 0, sizeof(unsigned) * (size_t)(n > 0 ? n : 1), s) != cudaSuccess)
    return DSMC_ERR_CUDA;
  k_collide_vhs<<<blocks, sh.threads, 0, s>>>(a);
  count_launches(c, 1);
  return cudaGetLastError() == cudaSuccess ? 0 : record(c, DSMC_ERR_CUDA, "collide_vhs: launch failed");
}

// Failure-detection self test: every block but block 0 enters the grid
// barrier; block 0 never arrives, so the others' bounded waits run out and
// record DSMC_ERR_TIMEOUT.  No trap, no unbounded spin.
__global__ void k_selftest_barrier(unsigned* bar, int* status, uint64_t limit_ns) {
  if (blockIdx.x == 0) return;
  grid_barrier(bar, status, limit_ns);
}

// Failure-detection self test of the pair-dependency wait: one thread waits
// for a done stamp that nothing ever sets (word 0 of the zeroed barrier
// words); the bounded wait must record DSMC_ERR_TIMEOUT and return.
__global__ void k_selftest_deps(unsigned* bar, int* status, uint64_t limit_ns) {
  if (threadIdx.x == 0) wait_deps(bar, 0, 0, 1u, bar + 2, status, limit_ns);
}

int launch_selftest_deps(Ctx* c, uint64_t limit_ns, cudaStream_t s) {
  unsigned* bar = barrier_ptr(c);
  if (cudaMemsetAsync(bar, 0, 4 * sizeof(unsigned), s) != cudaSuccess) return DSMC_ERR_CUDA;
  k_selftest_deps<<<1, 32, 0, s>>>(bar, status_ptr(c), limit_ns);
  count_launches(c, 1);
  return cudaGetLastError() == cudaSuccess ? 0 : record(c, DSMC_ERR_CUDA, "selftest_deps: launch failed");
}

int launch_selftest_barrier(Ctx* c, uint64_t limit_ns, cudaStream_t s) {
  if (cudaMemsetAsync(barrier_ptr(c), 0, 4 * sizeof(unsigned), s) != cudaSuccess) return DSMC_ERR_CUDA;
  unsigned* bar = barrier_ptr(c);
  int* st = status_ptr(c);
  void* args[] = {&bar, &st, &limit_ns};
  if (cudaLaunchCooperativeKernel((const void*)k_selftest_barrier, dim3(4), dim3(32), args, 0, s) != cudaSuccess)
    return record(c, DSMC_ERR_CUDA, "selftest_barrier: launch failed");
  count_launches(c, 1);
  return 0;
}

}  // namespace dsmc
