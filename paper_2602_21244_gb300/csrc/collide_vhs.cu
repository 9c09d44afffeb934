// VHS isotropic scatter with the centre-of-mass update (Sec. 2.1, 2.3).
//
// One persistent cooperative launch walks the rounds of the step: the pairs
// of a round are disjoint, so its threads update them independently; a
// bounded grid barrier separates rounds.  Velocities are read and written
// through L2 (ld/st .cg) so that a round sees the previous round's writes
// from other SMs.
#include "internal.cuh"

namespace dsmc {

struct VhsArgs {
  uint64_t seed, step;
  const uint64_t* step_dev;
  const int4* pairs;
  const int32_t* ro;
  const dsmc_select_info_t* info;
  double *vx, *vy, *vz;
  unsigned* bar;
  int* status;
};

__global__ void __launch_bounds__(256) k_collide_vhs(VhsArgs a) {
  if (a.step_dev) a.step = *a.step_dev;
  const int R = a.info->n_rounds;
  const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
  for (int r = 0; r < R; ++r) {
    const int32_t beg = a.ro[r], end = a.ro[r + 1];
    for (int64_t p = beg + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < end; p += nthr) {
      const int4 q = a.pairs[p];
      const double xi = __ldcg(a.vx + q.x), yi = __ldcg(a.vy + q.x), zi = __ldcg(a.vz + q.x);
      const double xj = __ldcg(a.vx + q.y), yj = __ldcg(a.vy + q.y), zj = __ldcg(a.vz + q.y);
      const double dx = xi - xj, dy = yi - yj, dz = zi - zj;
      const double g = sqrt(dx * dx + dy * dy + dz * dz);
      const u32x4 w = draw(a.seed, (uint32_t)q.w, (uint32_t)q.z, a.step, TAG_ISO);
      const double c = 2.0 * u53(w.x, w.y) - 1.0;
      const double s = sqrt(1.0 - c * c);
      double se, ce;
      sincos(2.0 * DSMC_PI * u53(w.z, w.w), &se, &ce);
      const double rx = g * c, ry = g * s * ce, rz = g * s * se;
      const double cx = 0.5 * (xi + xj), cy = 0.5 * (yi + yj), cz = 0.5 * (zi + zj);
      __stcg(a.vx + q.x, cx + 0.5 * rx); __stcg(a.vy + q.x, cy + 0.5 * ry); __stcg(a.vz + q.x, cz + 0.5 * rz);
      __stcg(a.vx + q.y, cx - 0.5 * rx); __stcg(a.vy + q.y, cy - 0.5 * ry); __stcg(a.vz + q.y, cz - 0.5 * rz);
    }
    if (r + 1 < R && !grid_barrier(a.bar, a.status, kBarrierLimitNs)) return;
  }
}

int cooperative_blocks(Ctx* c, const void* kernel, int threads, size_t smem) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
      per_sm < 1)
    return 0;
  return per_sm * sm_count(c);
}

// resident blocks per SM of the VHS collide at a block size (0 on failure)
int occupancy_collide_vhs(int threads) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k_collide_vhs, threads, 0) != cudaSuccess)
    return 0;
  return per_sm;
}

int launch_collide_vhs(Ctx* c, const dsmc_gas_t& gas, uint64_t step, const int32_t* pairs,
                       const int32_t* ro, const dsmc_select_info_t* info, double* vx,
                       double* vy, double* vz, cudaStream_t s) {
  const Shape sh = shape_or_default(c, DSMC_TUNE_COLLIDE_VHS);
  const int occ = occupancy_collide_vhs(sh.threads);
  if (occ < 1) return record(c, DSMC_ERR_CUDA, "collide_vhs: occupancy query failed");
  const int blocks = sm_count(c) * (sh.blocks_per_sm > 0 && sh.blocks_per_sm < occ ? sh.blocks_per_sm : occ);
  VhsArgs a{gas.seed, step, graph_step_ptr(c), (const int4*)pairs, ro, info, vx, vy, vz, barrier_ptr(c), status_ptr(c)};
  if (cudaMemsetAsync(a.bar, 0, 4 * sizeof(unsigned), s) != cudaSuccess) return DSMC_ERR_CUDA;
  void* args[] = {&a};
  if (cudaLaunchCooperativeKernel((const void*)k_collide_vhs, dim3(blocks), dim3(sh.threads), args, 0, s) !=
      cudaSuccess)
    return record(c, DSMC_ERR_CUDA, "collide_vhs: cooperative launch failed");
  count_launches(c, 1);
  return 0;
}

// Failure-detection self test: every block but block 0 enters the grid
// barrier; block 0 never arrives, so the others' bounded waits run out and
// record DSMC_ERR_TIMEOUT.  No trap, no unbounded spin.
__global__ void k_selftest_barrier(unsigned* bar, int* status, uint64_t limit_ns) {
  if (blockIdx.x == 0) return;
  grid_barrier(bar, status, limit_ns);
}

int launch_selftest_timeout(Ctx* c, int which, uint64_t limit_ns, cudaStream_t s);

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
