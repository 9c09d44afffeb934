// C ABI of the DSMC library: context, status word, argument checks, the
// whole collision step and its host-buffer variant.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "internal.cuh"

namespace dsmc {

struct Ctx {
  int device = 0;
  int sms = 0;
  int* d_status = nullptr;    // device status word
  unsigned* d_bar = nullptr;  // grid-barrier words
  int* h_status = nullptr;    // pinned mirror
  char err[256] = {0};
  // dsmc_ctx_reserve buffers for dsmc_step_host
  int32_t r_n = 0, r_cells = 0;
  int64_t r_cap = 0;
  bool r_sg_ready = false;
  void* r_mem = nullptr;
  size_t r_bytes = 0;
  dsmc_step_buffers_t rb = {};
  double* r_T = nullptr;
  void* r_host_info = nullptr;
  // dsmc_step_host: a side stream for the copies that overlap the step
  cudaStream_t r_side = nullptr;
  // dsmc_step: a side stream for the cell moments, which run beside the
  // selection (both only read the sorted velocities)
  cudaStream_t f_side = nullptr;
  cudaEvent_t f_ev[2] = {nullptr, nullptr};
  cudaEvent_t r_ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  int64_t launches = 0;
  int64_t graph_launches = 0;
  // step graph
  cudaGraphExec_t graph_exec = nullptr;
  bool capturing = false;
  // launch shapes (dsmc_tune_set); 0 = built-in
  int tune_threads[DSMC_TUNE_KERNELS] = {0};
  int tune_bps[DSMC_TUNE_KERNELS] = {0};
};

int record(Ctx* c, int code, const char* msg) {
  if (c && msg) snprintf(c->err, sizeof(c->err), "%s", msg);
  return code;
}
int* status_ptr(Ctx* c) { return c->d_status; }
// grid-barrier words: one slot for direct calls, another for graph replays,
// so that a replay and a direct call on another stream do not share counters
unsigned* barrier_ptr(Ctx* c) { return c->capturing ? c->d_bar + 32 : c->d_bar; }
// work counters: words 40-41 for direct calls, 48-49 for graph replays
unsigned* work_ptr(Ctx* c) { return c->capturing ? c->d_bar + 48 : c->d_bar + 40; }
int sm_count(Ctx* c) { return c->sms; }
Shape tune_shape(Ctx* c, int k) { return Shape{c->tune_threads[k], c->tune_bps[k]}; }
void count_launches(Ctx* c, int k) { c->launches += k; }
// the step index of a graph replay lives 64 bytes into the barrier block
static uint64_t* step_slot(Ctx* c) { return (uint64_t*)((char*)c->d_bar + 64); }
const uint64_t* graph_step_ptr(Ctx* c) { return c->capturing ? step_slot(c) : nullptr; }

__global__ void k_set_step(uint64_t* slot, uint64_t step) { *slot = step; }

// built-in launch shapes; blocks_per_sm 0 = as many as the occupancy allows
ShapeInfo shape_info(int k) {
  switch (k) {
    case DSMC_TUNE_GATHER: return ShapeInfo{256, 16, 1024};
    case DSMC_TUNE_MOMENTS: return ShapeInfo{256, 4, 256};
    case DSMC_TUNE_MOMENT_MATCH: return ShapeInfo{256, 3, 256};
    case DSMC_TUNE_COLLIDE_VHS: return ShapeInfo{256, 0, 256};
    case DSMC_TUNE_COLLIDE_JAGER: return ShapeInfo{128, 0, 128};
    case DSMC_TUNE_JAGER_CHI: return ShapeInfo{128, 64, 128};
    case DSMC_TUNE_COLLIDE_TABLE: return ShapeInfo{256, 0, 256};
    default: return ShapeInfo{0, 0, 0};
  }
}

// Candidate shapes of one kernel: block sizes up to the kernel's limit with
// at most 2048 threads and 32 blocks per SM (the chi batch grid-strides over up to
// 64 blocks per SM); for the persistent collides
// the full occupancy at each block size and half of it.
static int tune_candidates(int k, dsmc_tune_entry_t* out, int cap) {
  int n = 0;
  auto push = [&](int t, int b) {
    if (n < cap && out) out[n] = dsmc_tune_entry_t{k, t, b, 0.f};
    ++n;
  };
  switch (k) {
    case DSMC_TUNE_GATHER:
      for (int t : {128, 256, 512})
        for (int b : {2, 4, 8, 16})
          if (t * b <= 2048) push(t, b);
      break;
    case DSMC_TUNE_MOMENTS:
    case DSMC_TUNE_MOMENT_MATCH:
      // block size fixed (256 threads); up to four blocks resident per SM
      for (int b : {1, 2, 3, 4}) push(256, b);
      break;
    case DSMC_TUNE_COLLIDE_VHS:
    case DSMC_TUNE_COLLIDE_JAGER:
    case DSMC_TUNE_COLLIDE_TABLE: {
      const bool wide = k != DSMC_TUNE_COLLIDE_JAGER;
      for (int t : {32, 64, 128, 256}) {
        if (t > shape_info(k).max_threads || (wide && t < 64)) continue;
        const int occ = k == DSMC_TUNE_COLLIDE_VHS ? occupancy_collide_vhs(t)
                        : k == DSMC_TUNE_COLLIDE_JAGER ? occupancy_collide_jager(t) : occupancy_collide_table(t);
        if (occ < 1) continue;
        push(t, occ > 32 ? 32 : occ);
        if (occ / 2 >= 1) push(t, occ / 2 > 32 ? 32 : occ / 2);
      }
      break;
    }
    case DSMC_TUNE_JAGER_CHI:
      for (int t : {64, 128})
        for (int b : {8, 16, 32, 64}) push(t, b);
      break;
    default: break;
  }
  return n;
}

}  // namespace dsmc

using dsmc::Ctx;
struct dsmc_ctx : dsmc::Ctx {};

static inline cudaStream_t S(void* s) { return (cudaStream_t)s; }

#define CHECK_CTX(c) \
  do { if (!(c)) return DSMC_ERR_ARG; } while (0)
#define REQUIRE(c, cond, msg) \
  do { if (!(cond)) return dsmc::record((c), DSMC_ERR_ARG, (msg)); } while (0)

extern "C" {

int dsmc_abi_version(void) { return DSMC_ABI_VERSION; }

int dsmc_ctx_create(dsmc_ctx_t** out, int device) {
  if (!out) return DSMC_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return DSMC_ERR_CUDA;
  if (cudaSetDevice(device) != cudaSuccess) return DSMC_ERR_CUDA;
  dsmc_ctx* c = new dsmc_ctx();
  c->device = device;
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
  bool ok = cudaMalloc(&c->d_status, 256) == cudaSuccess &&
            cudaMalloc(&c->d_bar, 256) == cudaSuccess &&
            cudaMallocHost(&c->h_status, 256) == cudaSuccess &&
            cudaMemset(c->d_status, 0, 256) == cudaSuccess &&
            cudaMemset(c->d_bar, 0, 256) == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess &&
            cudaStreamCreateWithFlags(&c->f_side, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&c->f_ev[0], cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&c->f_ev[1], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    dsmc_ctx_destroy(c);
    return DSMC_ERR_CUDA;
  }
  *out = c;
  return DSMC_OK;
}

void dsmc_ctx_destroy(dsmc_ctx_t* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  if (c->d_status) cudaFree(c->d_status);
  if (c->d_bar) cudaFree(c->d_bar);
  if (c->h_status) cudaFreeHost(c->h_status);
  if (c->r_mem) cudaFree(c->r_mem);
  if (c->r_host_info) cudaFreeHost(c->r_host_info);
  for (cudaEvent_t e : c->r_ev)
    if (e) cudaEventDestroy(e);
  if (c->r_side) cudaStreamDestroy(c->r_side);
  for (cudaEvent_t e : c->f_ev)
    if (e) cudaEventDestroy(e);
  if (c->f_side) cudaStreamDestroy(c->f_side);
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  delete c;
}

int dsmc_ctx_sync_status(dsmc_ctx_t* c, void* stream) {
  CHECK_CTX(c);
  if (cudaMemcpyAsync(c->h_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, S(stream)) !=
          cudaSuccess ||
      cudaMemsetAsync(c->d_status, 0, sizeof(int), S(stream)) != cudaSuccess ||
      cudaStreamSynchronize(S(stream)) != cudaSuccess)
    return dsmc::record(c, DSMC_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
  return *c->h_status;
}

const char* dsmc_last_error(dsmc_ctx_t* c) { return c ? c->err : "null context"; }

int64_t dsmc_ctx_launch_count(dsmc_ctx_t* c) { return c ? c->launches : -1; }

size_t dsmc_sort_workspace_size(int32_t n, int32_t n_cells) { return dsmc::sort_ws(n, n_cells); }

int dsmc_sort_cells(dsmc_ctx_t* c, int32_t n, int32_t n_cells, const int32_t* cell_id,
                    const double* vx, const double* vy, const double* vz, int32_t* perm,
                    int32_t* cell_start, double* svx, double* svy, double* svz, void* ws,
                    size_t ws_bytes, void* stream) {
  CHECK_CTX(c);
  REQUIRE(c, n >= 0 && n_cells >= 1, "sort: n < 0 or n_cells < 1");
  REQUIRE(c, cell_start && ws, "sort: null cell_start or workspace");
  REQUIRE(c, n == 0 || (cell_id && vx && vy && vz && perm && svx && svy && svz), "sort: null array");
  return dsmc::launch_sort(c, n, n_cells, cell_id, vx, vy, vz, perm, cell_start, svx, svy, svz,
                           ws, ws_bytes, S(stream));
}

int dsmc_cell_moments(dsmc_ctx_t* c, int32_t n_cells, const int32_t* cell_start,
                      const double* vx, const double* vy, const double* vz, double* mom,
                      void* stream) {
  CHECK_CTX(c);
  REQUIRE(c, n_cells >= 0 && cell_start && mom, "moments: bad arguments");
  return dsmc::launch_moments(c, n_cells, cell_start, vx, vy, vz, mom, S(stream));
}

int dsmc_sigma_g_max_init(dsmc_ctx_t* c, const dsmc_gas_t* gas, int32_t n_cells,
                          const double* T_cell, double factor, double* sgmax, void* stream) {
  CHECK_CTX(c);
  REQUIRE(c, gas && T_cell && sgmax && n_cells >= 0 && factor > 0, "sigma_g_max_init: bad arguments");
  return dsmc::launch_sgmax_init(c, *gas, n_cells, T_cell, factor, sgmax, S(stream));
}

size_t dsmc_select_workspace_size(int32_t n, int32_t n_cells, int64_t capacity) {
  return dsmc::select_ws(n, n_cells, capacity);
}

static int check_gas(Ctx* c, const dsmc_gas_t* gas) {
  REQUIRE(c, gas, "null gas");
  REQUIRE(c, gas->mass > 0 && gas->dt > 0 && gas->fn_over_vc > 0, "gas: mass, dt, fn_over_vc > 0");
  REQUIRE(c, gas->model == 0 || gas->model == 1, "gas: model must be 0 or 1");
  REQUIRE(c, gas->model == 1 || (gas->d_ref > 0 && gas->T_ref > 0 && gas->omega > 0 && gas->omega < 2.5),
          "gas: VHS needs d_ref, T_ref > 0, 0 < omega < 2.5");
  REQUIRE(c, gas->model == 0 || gas->b_max > 0, "gas: constant cross section needs b_max > 0");
  return 0;
}

int dsmc_select_pairs_ordered(dsmc_ctx_t* c, const dsmc_gas_t* gas, int32_t n, int32_t n_cells,
                              const int32_t* cell_start, const double* vx, const double* vy,
                              const double* vz, double* sgmax, uint64_t step, int64_t capacity,
                              int32_t* pairs, uint32_t* deps, int32_t* round_offsets, dsmc_select_info_t* info,
                              int32_t order, void* ws, size_t ws_bytes, void* stream) {
  CHECK_CTX(c);
  if (int rc = check_gas(c, gas)) return rc;
  REQUIRE(c, n >= 0 && n_cells >= 1 && capacity >= 0, "select: bad sizes");
  REQUIRE(c, cell_start && sgmax && round_offsets && info && ws, "select: null pointer");
  REQUIRE(c, capacity == 0 || (pairs && deps), "select: null pairs or deps");
  REQUIRE(c, order == DSMC_ORDER_ROUNDS || order == DSMC_ORDER_LEVELS, "select: bad order");
  return dsmc::launch_select(c, *gas, n, n_cells, cell_start, vx, vy, vz, sgmax, step, capacity,
                             pairs, deps, round_offsets, info, ws, ws_bytes, order, S(stream));
}

int dsmc_select_pairs(dsmc_ctx_t* c, const dsmc_gas_t* gas, int32_t n, int32_t n_cells,
                      const int32_t* cell_start, const double* vx, const double* vy,
                      const double* vz, double* sgmax, uint64_t step, int64_t capacity,
                      int32_t* pairs, uint32_t* deps, int32_t* round_offsets, dsmc_select_info_t* info,
                      void* ws, size_t ws_bytes, void* stream) {
  return dsmc_select_pairs_ordered(c, gas, n, n_cells, cell_start, vx, vy, vz, sgmax, step, capacity, pairs,
                                   deps, round_offsets, info, DSMC_ORDER_ROUNDS, ws, ws_bytes, stream);
}

size_t dsmc_collide_workspace_size(int32_t n) { return dsmc::collide_ws(n); }

int dsmc_collide_vhs(dsmc_ctx_t* c, const dsmc_gas_t* gas, uint64_t step, int32_t n, const int32_t* pairs,
                     const uint32_t* deps, const int32_t* round_offsets, const dsmc_select_info_t* info,
                     double* vx, double* vy, double* vz, void* ws, size_t ws_bytes, void* stream) {
  CHECK_CTX(c);
  REQUIRE(c, gas && round_offsets && info && vx && vy && vz && ws && n >= 0, "collide_vhs: null pointer");
  return dsmc::launch_collide_vhs(c, *gas, step, n, pairs, deps, round_offsets, info, vx, vy, vz, ws, ws_bytes,
                                  S(stream));
}

static int check_pot(Ctx* c, const dsmc_potential_t* p, int n_nodes) {
  REQUIRE(c, p, "null potential");
  REQUIRE(c, p->kind >= 0 && p->kind <= 2, "potential: kind must be 0, 1 or 2");
  REQUIRE(c, n_nodes >= 8 && n_nodes <= 128, "potential: n_nodes must be in [8, 128]");
  REQUIRE(c, p->kind != 0 || p->R_eps > 0, "potential: Jager form needs R_eps > 0");
  REQUIRE(c, p->kind != 1 || p->d_hs > 0, "potential: hard sphere needs d_hs > 0");
  REQUIRE(c, p->kind != 2 || p->p > 0, "potential: inverse power needs p > 0");
  return 0;
}

int dsmc_jager_chi(dsmc_ctx_t* c, const dsmc_gas_t* gas, const dsmc_potential_t* pot,
                   int32_t n_nodes, int64_t n, const float* b, const float* g, float* chi,
                   void* stream) {
  CHECK_CTX(c);
  REQUIRE(c, gas && gas->mass > 0, "jager_chi: gas with mass > 0 required");
  if (int rc = check_pot(c, pot, n_nodes)) return rc;
  REQUIRE(c, n >= 0 && (n == 0 || (b && g && chi)), "jager_chi: bad arrays");
  return dsmc::launch_jager_chi(c, *gas, *pot, n_nodes, n, b, g, chi, S(stream));
}

int dsmc_transport_q2(dsmc_ctx_t* c, const dsmc_potential_t* pot, int32_t n_nodes, int32_t n_E,
                      const double* E_kelvin, double b_max_A, int32_t b_panels, double* q2, void* stream) {
  CHECK_CTX(c);
  if (int rc = check_pot(c, pot, n_nodes)) return rc;
  REQUIRE(c, n_E >= 0 && (n_E == 0 || (E_kelvin && q2)), "transport_q2: bad arrays");
  REQUIRE(c, b_max_A > 0 && b_panels >= 1 && b_panels <= 4096, "transport_q2: b_max > 0, b_panels in [1, 4096]");
  return dsmc::launch_transport_q2(c, *pot, n_nodes, n_E, E_kelvin, b_max_A, b_panels, q2, S(stream));
}

size_t dsmc_transport_workspace_size(int32_t n_T, int32_t x_panels) {
  if (n_T < 0 || x_panels < 1) return 0;
  return dsmc::transport_ws(n_T, x_panels);
}

int dsmc_transport_viscosity(dsmc_ctx_t* c, const dsmc_gas_t* gas, const dsmc_potential_t* pot, int32_t n_nodes,
                             int32_t n_T, const double* T_kelvin, double b_max_A, int32_t b_panels,
                             int32_t x_panels, double* omega22, double* mu, void* ws, size_t ws_bytes,
                             void* stream) {
  CHECK_CTX(c);
  REQUIRE(c, gas && gas->mass > 0, "transport_viscosity: gas with mass > 0 required");
  if (int rc = check_pot(c, pot, n_nodes)) return rc;
  REQUIRE(c, n_T >= 0 && (n_T == 0 || (T_kelvin && omega22 && mu && ws)), "transport_viscosity: bad arrays");
  REQUIRE(c, b_max_A > 0 && b_panels >= 1 && b_panels <= 4096 && x_panels >= 1 && x_panels <= 1024,
          "transport_viscosity: b_max > 0, b_panels in [1, 4096], x_panels in [1, 1024]");
  return dsmc::launch_transport_viscosity(c, *gas, *pot, n_nodes, n_T, T_kelvin, b_max_A, b_panels, x_panels,
                                          omega22, mu, ws, ws_bytes, S(stream));
}

size_t dsmc_chi_mlp_packed_size(void) { return dsmc::chi_mlp_packed_size(); }

int dsmc_chi_mlp_pack(dsmc_ctx_t* c, const uint16_t* w_bits, void* packed, void* stream) {
  CHECK_CTX(c);
  REQUIRE(c, w_bits && packed, "chi_mlp_pack: null pointer");
  REQUIRE(c, ((uintptr_t)packed & 15u) == 0, "chi_mlp_pack: packed buffer must be 16-byte aligned");
  return dsmc::launch_chi_mlp_pack(c, w_bits, packed, S(stream));
}

int dsmc_chi_mlp_forward(dsmc_ctx_t* c, const void* packed, const float* bias, int64_t n, const float* x, float* y,
                         float* chi, void* stream) {
  CHECK_CTX(c);
  REQUIRE(c, packed && bias && n >= 0 && (n == 0 || (x && (y || chi))), "chi_mlp_forward: bad arguments");
  REQUIRE(c, ((uintptr_t)packed & 15u) == 0, "chi_mlp_forward: packed buffer must be 16-byte aligned");
  return dsmc::launch_chi_mlp_forward(c, packed, bias, n, x, y, chi, S(stream));
}

int dsmc_chi_mlp_table(dsmc_ctx_t* c, const void* packed, const float* bias, int32_t nb, int32_t nE, float* table,
                       void* stream) {
  CHECK_CTX(c);
  REQUIRE(c, packed && bias && table && nb >= 2 && nE >= 2 && (int64_t)nb * nE <= (1ll << 31),
          "chi_mlp_table: bad arguments");
  REQUIRE(c, ((uintptr_t)packed & 15u) == 0, "chi_mlp_table: packed buffer must be 16-byte aligned");
  return dsmc::launch_chi_mlp_table(c, packed, bias, nb, nE, table, S(stream));
}

int dsmc_collide_jager(dsmc_ctx_t* c, const dsmc_gas_t* gas, const dsmc_potential_t* pot,
                       int32_t n_nodes, uint64_t step, int32_t n, const int32_t* pairs, const uint32_t* deps,
                       const int32_t* round_offsets, const dsmc_select_info_t* info,
                       double* vx, double* vy, double* vz, float* chi_out, void* ws, size_t ws_bytes,
                       void* stream) {
  CHECK_CTX(c);
  REQUIRE(c, gas && gas->b_max > 0, "collide_jager: gas with b_max > 0 required");
  if (int rc = check_pot(c, pot, n_nodes)) return rc;
  REQUIRE(c, round_offsets && info && vx && vy && vz && ws && n >= 0, "collide_jager: null pointer");
  return dsmc::launch_collide_jager(c, *gas, *pot, n_nodes, step, n, pairs, deps, round_offsets, info, vx,
                                    vy, vz, chi_out, ws, ws_bytes, S(stream));
}

static int check_table(Ctx* c, const dsmc_chi_table_t* t) {
  REQUIRE(c, t && t->chi, "null chi table");
  REQUIRE(c, t->nb >= 2 && t->nb <= 4096 && t->nE >= 2 && t->nE <= 4096, "chi table: nb, nE must be 2..4096");
  REQUIRE(c, t->lnE_max > t->lnE_min, "chi table: lnE_max must exceed lnE_min");
  return 0;
}

int dsmc_chi_table_build(dsmc_ctx_t* c, const dsmc_gas_t* gas, const dsmc_potential_t* pot, int32_t n_nodes,
                         int32_t nb, int32_t nE, double lnE_min, double lnE_max, float* table, void* stream) {
  CHECK_CTX(c);
  REQUIRE(c, gas && gas->mass > 0 && gas->b_max > 0, "chi_table: gas with mass and b_max > 0 required");
  if (int rc = check_pot(c, pot, n_nodes)) return rc;
  const dsmc_chi_table_t t{table, nb, nE, lnE_min, lnE_max};
  if (int rc = check_table(c, &t)) return rc;
  return dsmc::launch_chi_table(c, *gas, *pot, n_nodes, nb, nE, lnE_min, lnE_max, table, S(stream));
}

int dsmc_collide_table(dsmc_ctx_t* c, const dsmc_gas_t* gas, const dsmc_chi_table_t* table, uint64_t step,
                       int32_t n, const int32_t* pairs, const uint32_t* deps, const int32_t* round_offsets,
                       const dsmc_select_info_t* info, double* vx, double* vy, double* vz, float* chi_out,
                       void* ws, size_t ws_bytes, void* stream) {
  CHECK_CTX(c);
  REQUIRE(c, gas && gas->mass > 0, "collide_table: gas with mass > 0 required");
  if (int rc = check_table(c, table)) return rc;
  REQUIRE(c, round_offsets && info && vx && vy && vz && ws && n >= 0, "collide_table: null pointer");
  return dsmc::launch_collide_table(c, *gas, *table, step, n, pairs, deps, round_offsets, info, vx, vy, vz, chi_out,
                                    ws, ws_bytes, S(stream));
}

static int check_mlp(Ctx* c, const dsmc_mlp_t* m) {
  REQUIRE(c, m, "null mlp");
  REQUIRE(c, m->width == 128 && m->d_out == 3 && (m->d_in == 6 || m->d_in == 8) &&
                 m->n_hidden >= 1 && m->n_hidden <= 4 && (m->act == 0 || m->act == 1),
          "mlp: supported shape is d_in 6|8, width 128, 1..4 hidden layers, d_out 3, act 0|1");
  REQUIRE(c, m->sigma_v > 0 && m->T_ref > 0 && m->eps >= 0, "mlp: sigma_v, T_ref > 0, eps >= 0");
  return 0;
}

int dsmc_collide_neural(dsmc_ctx_t* c, const dsmc_gas_t* gas, const dsmc_mlp_t* mlp,
                        const uint16_t* w, const float* bias, uint64_t step,
                        const double* mom_pre, int32_t n, const int32_t* pairs, const uint32_t* deps,
                        const int32_t* round_offsets, const dsmc_select_info_t* info,
                        double* vx, double* vy, double* vz, float* u_out, void* ws, size_t ws_bytes,
                        void* stream) {
  CHECK_CTX(c);
  REQUIRE(c, gas, "collide_neural: null gas");
  if (int rc = check_mlp(c, mlp)) return rc;
  REQUIRE(c, w && bias && mom_pre && round_offsets && info && vx && vy && vz && ws && n >= 0,
          "collide_neural: null pointer");
  return dsmc::launch_collide_neural(c, *gas, *mlp, w, bias, step, mom_pre, n, pairs, deps, round_offsets,
                                     info, vx, vy, vz, u_out, ws, ws_bytes, S(stream));
}

int dsmc_mlp_forward(dsmc_ctx_t* c, const dsmc_mlp_t* mlp, const uint16_t* w, const float* bias,
                     int64_t n, const float* x, float* y, void* stream) {
  CHECK_CTX(c);
  if (int rc = check_mlp(c, mlp)) return rc;
  REQUIRE(c, w && bias && n >= 0 && (n == 0 || (x && y)), "mlp_forward: bad arguments");
  return dsmc::launch_mlp_forward(c, *mlp, w, bias, n, x, y, S(stream));
}

int dsmc_tc_selftest(dsmc_ctx_t* c, int32_t N, int32_t K, int32_t layout, const uint16_t* A,
                     const uint16_t* B, float* D, void* stream) {
  CHECK_CTX(c);
  REQUIRE(c, N >= 16 && N <= 256 && N % 16 == 0 && K >= 16 && K <= 128 && K % 16 == 0,
          "tc_selftest: N in [16,256], K in [16,128], multiples of 16");
  REQUIRE(c, layout >= 0 && layout <= 15 && !((layout & 8) && (layout & 1)),
          "tc_selftest: layout in [0, 15], A in tensor memory is K-major");
  REQUIRE(c, A && B && D, "tc_selftest: null pointer");
  return dsmc::launch_tc_selftest(c, N, K, layout, A, B, D, S(stream));
}

int dsmc_selftest_timeout(dsmc_ctx_t* c, int32_t which, uint64_t limit_ns, void* stream) {
  CHECK_CTX(c);
  REQUIRE(c, which >= 0 && which <= 2 && limit_ns > 0 && limit_ns <= 2000000000ull,
          "selftest_timeout: which 0|1|2, 0 < limit_ns <= 2e9");
  if (which == 2) return dsmc::launch_selftest_deps(c, limit_ns, S(stream));
  return which == 0 ? dsmc::launch_selftest_barrier(c, limit_ns, S(stream))
                    : dsmc::launch_selftest_mbar(c, limit_ns, S(stream));
}

int dsmc_selftest_math(dsmc_ctx_t* c, int32_t which, int64_t n, const double* x, double* y, void* stream) {
  CHECK_CTX(c);
  REQUIRE(c, which >= 0 && which <= 3 && n >= 0 && (n == 0 || (x && y)), "selftest_math: which 0..3, n >= 0, x, y");
  return dsmc::launch_selftest_math(c, which, n, x, y, S(stream));
}

int64_t dsmc_selftest_peak_ops(int32_t which, int32_t iters) {
  if (which < 0 || which > 3 || iters < 1) return -1;
  return dsmc::peak_ops_per_thread(which, iters);
}

int dsmc_selftest_peak(dsmc_ctx_t* c, int32_t which, int32_t blocks, int32_t threads, int32_t iters, float* sink,
                       void* stream) {
  CHECK_CTX(c);
  REQUIRE(c, which >= 0 && which <= 3 && blocks >= 1 && threads >= 32 && threads <= 256 && threads % 32 == 0 &&
                 iters >= 1 && sink,
          "selftest_peak: which 0..3, blocks >= 1, threads a multiple of 32 up to 256, iters >= 1, sink");
  return dsmc::launch_peak(c, which, blocks, threads, iters, sink, S(stream));
}

int dsmc_moment_match(dsmc_ctx_t* c, int32_t n_cells, const int32_t* cell_start,
                      const double* mom_pre, double* vx, double* vy, double* vz, void* stream) {
  CHECK_CTX(c);
  REQUIRE(c, n_cells >= 0 && cell_start && mom_pre, "moment_match: bad arguments");
  return dsmc::launch_moment_match(c, n_cells, cell_start, mom_pre, vx, vy, vz, S(stream));
}

int dsmc_harvest_jager(dsmc_ctx_t* c, const dsmc_gas_t* gas, const dsmc_potential_t* pot,
                       int32_t n_nodes, int64_t n, const double* vi, const double* vj,
                       const double* b, const double* eps, double* vio, double* vjo,
                       void* stream) {
  CHECK_CTX(c);
  REQUIRE(c, gas && gas->mass > 0, "harvest: gas with mass > 0 required");
  if (int rc = check_pot(c, pot, n_nodes)) return rc;
  REQUIRE(c, n >= 0 && (n == 0 || (vi && vj && b && eps && vio && vjo)), "harvest: bad arrays");
  return dsmc::launch_harvest_jager(c, *gas, *pot, n_nodes, n, vi, vj, b, eps, vio, vjo, S(stream));
}

// ---------------------------------------------------------------- training
static int check_train(Ctx* c, const dsmc_mlp_t* mlp, int64_t n) {
  if (int rc = check_mlp(c, mlp)) return rc;
  REQUIRE(c, mlp->d_in == 8 && mlp->n_hidden == 3, "train: d_in 8 and 3 hidden layers");
  REQUIRE(c, n >= 0 && n % 16 == 0, "train: n_pairs must be a multiple of 16 (pseudo-cells)");
  return 0;
}

int32_t dsmc_mlp_param_count(const dsmc_mlp_t* mlp) {
  if (!mlp) return -1;
  const int32_t w = mlp->width * mlp->d_in + (mlp->n_hidden - 1) * mlp->width * mlp->width + mlp->d_out * mlp->width;
  return w + mlp->n_hidden * mlp->width + mlp->d_out;
}

size_t dsmc_train_workspace_size(dsmc_ctx_t* c) { return c ? dsmc::train_ws(c->sms) : 0; }

int dsmc_neural_operator_forward(dsmc_ctx_t* c, const dsmc_mlp_t* mlp, const float* theta, uint64_t seed,
                                 uint64_t t, int64_t n, const double* vi, const double* vj, const double* T,
                                 double* vi_new, double* vj_new, void* stream) {
  CHECK_CTX(c);
  if (int rc = check_train(c, mlp, n)) return rc;
  REQUIRE(c, theta && (n == 0 || (vi && vj && T && vi_new && vj_new)), "operator_forward: null pointer");
  if (n == 0) return 0;
  return dsmc::launch_train(c, *mlp, 0, seed, t, n, theta, vi, vj, T, nullptr, nullptr, nullptr, nullptr,
                            vi_new, vj_new, nullptr, nullptr, nullptr, 0, S(stream));
}

int dsmc_neural_operator_backward(dsmc_ctx_t* c, const dsmc_mlp_t* mlp, const float* theta, uint64_t seed,
                                  uint64_t t, int64_t n, const double* vi, const double* vj, const double* T,
                                  const double* g_vi, const double* g_vj, float* grad, void* ws, size_t ws_bytes,
                                  void* stream) {
  CHECK_CTX(c);
  if (int rc = check_train(c, mlp, n)) return rc;
  REQUIRE(c, theta && grad && ws && (n == 0 || (vi && vj && T && g_vi && g_vj)), "operator_backward: null pointer");
  return dsmc::launch_train(c, *mlp, 1, seed, t, n, theta, vi, vj, T, nullptr, nullptr, g_vi, g_vj, nullptr,
                            nullptr, grad, nullptr, ws, ws_bytes, S(stream));
}

int dsmc_train_loss_grad(dsmc_ctx_t* c, const dsmc_mlp_t* mlp, const float* theta, uint64_t seed, uint64_t t,
                         int64_t n, const double* vi, const double* vj, const double* T, const double* vi_target,
                         const double* vj_target, float* grad, double* loss, void* ws, size_t ws_bytes,
                         void* stream) {
  CHECK_CTX(c);
  if (int rc = check_train(c, mlp, n)) return rc;
  REQUIRE(c, theta && grad && loss && ws && (n == 0 || (vi && vj && T && vi_target && vj_target)),
          "train_loss_grad: null pointer");
  return dsmc::launch_train(c, *mlp, 2, seed, t, n, theta, vi, vj, T, vi_target, vj_target, nullptr, nullptr,
                            nullptr, nullptr, grad, loss, ws, ws_bytes, S(stream));
}

size_t dsmc_train_act_size(int64_t n) { return n > 0 ? dsmc::train_act_bytes(n) : 0; }

int dsmc_train_loss_grad_stored(dsmc_ctx_t* c, const dsmc_mlp_t* mlp, const float* theta, uint64_t seed, uint64_t t,
                                int64_t n, const double* vi, const double* vj, const double* T,
                                const double* vi_target, const double* vj_target, float* grad, double* loss,
                                void* ws, size_t ws_bytes, float* act, size_t act_bytes, void* stream) {
  CHECK_CTX(c);
  if (int rc = check_train(c, mlp, n)) return rc;
  REQUIRE(c, theta && grad && loss && ws && (n == 0 || (vi && vj && T && vi_target && vj_target && act)),
          "train_loss_grad_stored: null pointer");
  REQUIRE(c, act_bytes >= dsmc_train_act_size(n), "train_loss_grad_stored: activation buffer too small");
  return dsmc::launch_train(c, *mlp, 2, seed, t, n, theta, vi, vj, T, vi_target, vj_target, nullptr, nullptr,
                            nullptr, nullptr, grad, loss, ws, ws_bytes, S(stream), act);
}

int dsmc_adam_step(dsmc_ctx_t* c, int32_t n_params, int32_t n_weights, const float* grad, float* theta,
                   float* m, float* v, int64_t step, float lr, float beta1, float beta2, float eps,
                   uint16_t* weights_bf16, float* biases, void* stream) {
  CHECK_CTX(c);
  REQUIRE(c, n_params > 0 && n_weights >= 0 && n_weights <= n_params && step >= 1, "adam: bad sizes");
  REQUIRE(c, grad && theta && m && v, "adam: null pointer");
  return dsmc::launch_adam(c, n_weights, n_params - n_weights, grad, theta, m, v, weights_bf16, biases, lr, beta1,
                           beta2, eps, step, S(stream));
}

int dsmc_train_step(dsmc_ctx_t* c, const dsmc_mlp_t* mlp, float* theta, float* m, float* v, int64_t step,
                    float lr, uint64_t seed, int64_t n, const double* vi, const double* vj, const double* T,
                    const double* vi_target, const double* vj_target, float* grad, double* loss,
                    uint16_t* weights_bf16, float* biases, void* ws, size_t ws_bytes, void* stream) {
  int rc = dsmc_train_loss_grad(c, mlp, theta, seed, (uint64_t)step, n, vi, vj, T, vi_target, vj_target, grad,
                                loss, ws, ws_bytes, stream);
  if (rc) return rc;
  const int32_t np = dsmc_mlp_param_count(mlp);
  const int32_t nw = np - (mlp->n_hidden * mlp->width + mlp->d_out);
  return dsmc_adam_step(c, np, nw, grad, theta, m, v, step, lr, 0.9f, 0.999f, 1e-8f, weights_bf16, biases,
                        stream);
}

// ---------------------------------------------------------------- whole step
size_t dsmc_step_workspace_size(int32_t n, int32_t n_cells, int64_t capacity) {
  // the phases run one after another and share the workspace
  const size_t a = dsmc::sort_ws(n, n_cells), b = dsmc::select_ws(n, n_cells, capacity),
               d = dsmc::collide_ws(n);
  const size_t ab = a > b ? a : b, f = dsmc::fused_ws(n) > a ? dsmc::fused_ws(n) : a;
  const size_t abd = ab > d ? ab : d;
  return abd > f ? abd : f;
}

// the pair update of one step's path (after selection)
static int collide_step(dsmc_ctx_t* c, const dsmc_gas_t* gas, const dsmc_path_t* path,
                        const dsmc_step_buffers_t* B, uint64_t step, void* stream) {
  int rc = 0;
  switch (path->path) {
    case DSMC_PATH_VHS:
      rc = dsmc_collide_vhs(c, gas, step, B->n, B->pairs, B->deps, B->round_offsets, B->info, B->svx, B->svy,
                            B->svz, B->ws, B->ws_bytes, stream);
      break;
    case DSMC_PATH_JAGER:
      rc = dsmc_collide_jager(c, gas, path->pot, path->n_nodes, step, B->n, B->pairs, B->deps, B->round_offsets,
                              B->info, B->svx, B->svy, B->svz, nullptr, B->ws, B->ws_bytes, stream);
      break;
    case DSMC_PATH_NEURAL:
      rc = dsmc_collide_neural(c, gas, path->mlp, path->weights_bf16, path->biases, step, B->mom, B->n,
                               B->pairs, B->deps, B->round_offsets, B->info, B->svx, B->svy, B->svz,
                               nullptr, B->ws, B->ws_bytes, stream);
      break;
    case DSMC_PATH_TABLE:
      rc = dsmc_collide_table(c, gas, path->table, step, B->n, B->pairs, B->deps, B->round_offsets, B->info,
                              B->svx, B->svy, B->svz, nullptr, B->ws, B->ws_bytes, stream);
      break;
    default:
      return dsmc::record(c, DSMC_ERR_ARG, "step: unknown path");
  }
  return rc;
}

// The pair list's bucket order in a step: claim levels for the neural path,
// whose pair updates are long enough that the round structure's tail (the
// deep cells' last rounds, one dependency link each) sets its end; rounds
// for the others, whose short updates wait on fresher dependencies when the
// levels interleave the rounds.
static int32_t step_order(const dsmc_path_t* path) {
  return path->path == DSMC_PATH_NEURAL ? DSMC_ORDER_LEVELS : DSMC_ORDER_ROUNDS;
}

static int step_after_sort(dsmc_ctx_t* c, const dsmc_gas_t* gas, const dsmc_path_t* path,
                           const dsmc_step_buffers_t* B, uint64_t step, void* stream);

int dsmc_step(dsmc_ctx_t* c, const dsmc_gas_t* gas, const dsmc_path_t* path,
              const dsmc_step_buffers_t* B, uint64_t step, void* stream) {
  CHECK_CTX(c);
  REQUIRE(c, gas && path && B, "step: null argument");
  if (int rc = check_gas(c, gas)) return rc;
  REQUIRE(c, B->ws_bytes >= dsmc_step_workspace_size(B->n, B->n_cells, B->capacity),
          "step: workspace too small");
  int rc = dsmc_sort_cells(c, B->n, B->n_cells, B->cell_id, B->vx, B->vy, B->vz, B->perm,
                           B->cell_start, B->svx, B->svy, B->svz, B->ws, B->ws_bytes, stream);
  if (rc) return rc;
  return step_after_sort(c, gas, path, B, step, stream);
}

// the step from the sorted velocities on: moments (on the context's side
// stream, beside the selection: both only read the sorted velocities),
// selection, pair update, moment matching (after the moments have joined)
static int step_after_sort(dsmc_ctx_t* c, const dsmc_gas_t* gas, const dsmc_path_t* path,
                           const dsmc_step_buffers_t* B, uint64_t step, void* stream) {
  cudaStream_t s = S(stream);
  if (cudaEventRecord(c->f_ev[0], s) != cudaSuccess || cudaStreamWaitEvent(c->f_side, c->f_ev[0], 0) != cudaSuccess)
    return dsmc::record(c, DSMC_ERR_CUDA, "step: fork of the moments stream failed");
  int rc = dsmc_cell_moments(c, B->n_cells, B->cell_start, B->svx, B->svy, B->svz, B->mom, c->f_side);
  // the side stream joins the caller's stream whatever happens next
  const bool joined_ev = cudaEventRecord(c->f_ev[1], c->f_side) == cudaSuccess;
  if (!rc)
    rc = dsmc_select_pairs_ordered(c, gas, B->n, B->n_cells, B->cell_start, B->svx, B->svy, B->svz,
                                   B->sigma_g_max, step, B->capacity, B->pairs, B->deps, B->round_offsets,
                                   B->info, step_order(path), B->ws, B->ws_bytes, stream);
  if (!rc) rc = collide_step(c, gas, path, B, step, stream);
  const bool joined = joined_ev && cudaStreamWaitEvent(s, c->f_ev[1], 0) == cudaSuccess;
  if (rc) return rc;
  if (!joined) return dsmc::record(c, DSMC_ERR_CUDA, "step: join of the moments stream failed");
  return dsmc_moment_match(c, B->n_cells, B->cell_start, B->mom, B->svx, B->svy, B->svz, stream);
}

int dsmc_step_fused(dsmc_ctx_t* c, const dsmc_gas_t* gas, const dsmc_path_t* path,
                    const dsmc_step_buffers_t* B, uint64_t step, void* stream) {
  CHECK_CTX(c);
  REQUIRE(c, gas && path && B, "step_fused: null argument");
  if (int rc = check_gas(c, gas)) return rc;
  if (path->path != DSMC_PATH_VHS && path->path != DSMC_PATH_TABLE)
    return dsmc::record(c, DSMC_ERR_UNSUPPORTED, "step_fused: VHS and look-up paths only");
  if (path->path == DSMC_PATH_TABLE) {
    REQUIRE(c, gas->mass > 0, "step_fused: gas with mass > 0 required");
    if (int rc = check_table(c, path->table)) return rc;
  }
  REQUIRE(c, B->n >= 0 && B->n_cells >= 1 && B->capacity >= 0, "step_fused: bad sizes");
  REQUIRE(c, B->cell_start && B->ws && B->mom && B->sigma_g_max && B->info, "step_fused: null buffer");
  REQUIRE(c, B->n == 0 || (B->cell_id && B->vx && B->vy && B->vz && B->perm && B->svx && B->svy && B->svz),
          "step_fused: null array");
  REQUIRE(c, B->capacity == 0 || B->pairs, "step_fused: null pair buffer");
  REQUIRE(c, B->ws_bytes >= dsmc_step_workspace_size(B->n, B->n_cells, B->capacity),
          "step_fused: workspace too small");
  cudaStream_t s = S(stream);
  int rc = dsmc::launch_sort_keys(c, B->n, B->n_cells, B->cell_id, B->perm, B->cell_start, B->ws, B->ws_bytes, s);
  if (rc) return rc;
  return dsmc::launch_step_fused(c, *gas, path->path, path->table, step, B->n, B->n_cells, B->cell_start, B->perm,
                                 B->vx, B->vy, B->vz, B->svx, B->svy, B->svz, B->mom, B->sigma_g_max, B->pairs,
                                 B->capacity, B->info, B->ws, B->ws_bytes, s);
}

int dsmc_step_graph_capture(dsmc_ctx_t* c, const dsmc_gas_t* gas, const dsmc_path_t* path,
                            const dsmc_step_buffers_t* B, void* stream) {
  CHECK_CTX(c);
  REQUIRE(c, gas && path && B, "graph_capture: null argument");
  REQUIRE(c, stream, "graph_capture: needs a non-default stream");
  if (c->graph_exec) { cudaGraphExecDestroy(c->graph_exec); c->graph_exec = nullptr; }
  cudaStream_t s = S(stream);
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed) != cudaSuccess)
    return dsmc::record(c, DSMC_ERR_CUDA, "graph_capture: cudaStreamBeginCapture failed");
  c->capturing = true;
  const int64_t launches0 = c->launches;
  const int rc = dsmc_step(c, gas, path, B, 0, stream);
  c->capturing = false;
  c->graph_launches = c->launches - launches0;
  c->launches = launches0;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(s, &g);
  if (rc) { if (g) cudaGraphDestroy(g); return rc; }
  if (e != cudaSuccess || !g) return dsmc::record(c, DSMC_ERR_CUDA, "graph_capture: cudaStreamEndCapture failed");
  const cudaError_t ei = cudaGraphInstantiate(&c->graph_exec, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) { c->graph_exec = nullptr; return dsmc::record(c, DSMC_ERR_CUDA, "graph_capture: instantiate failed"); }
  return DSMC_OK;
}

int dsmc_step_graph_launch(dsmc_ctx_t* c, uint64_t step, void* stream) {
  CHECK_CTX(c);
  REQUIRE(c, c->graph_exec, "graph_launch: no captured step (dsmc_step_graph_capture)");
  dsmc::k_set_step<<<1, 1, 0, S(stream)>>>(dsmc::step_slot(c), step);
  if (cudaGraphLaunch(c->graph_exec, S(stream)) != cudaSuccess)
    return dsmc::record(c, DSMC_ERR_CUDA, "graph_launch: cudaGraphLaunch failed");
  c->launches += 1 + c->graph_launches;
  return DSMC_OK;
}

int dsmc_ctx_reserve(dsmc_ctx_t* c, int32_t n_max, int32_t n_cells, int64_t capacity) {
  CHECK_CTX(c);
  REQUIRE(c, n_max >= 0 && n_cells >= 1 && capacity >= 0, "reserve: bad sizes");
  if (c->r_mem) { cudaFree(c->r_mem); c->r_mem = nullptr; }
  const size_t n = (size_t)(n_max > 0 ? n_max : 1), nc = (size_t)n_cells;
  const size_t wsb = dsmc_step_workspace_size(n_max, n_cells, capacity);
  const size_t cap = (size_t)(capacity > 0 ? capacity : 1);
  size_t sizes[] = {4 * n, 8 * n, 8 * n, 8 * n, 4 * n, 4 * (nc + 1), 8 * n, 8 * n, 8 * n,
                    40 * nc, 8 * nc, 16 * cap,
                    4 * (DSMC_MAX_ROUNDS + 1), sizeof(dsmc_select_info_t), 8 * nc, wsb, 4 * cap};
  size_t total = 0;
  for (size_t s : sizes) total += dsmc::align256(s);
  if (cudaSetDevice(c->device) != cudaSuccess || cudaMalloc(&c->r_mem, total) != cudaSuccess)
    return dsmc::record(c, DSMC_ERR_CUDA, "reserve: cudaMalloc failed");
  if (!c->r_host_info && cudaMallocHost(&c->r_host_info, 64) != cudaSuccess)
    return dsmc::record(c, DSMC_ERR_CUDA, "reserve: cudaMallocHost failed");
  char* p = (char*)c->r_mem;
  void* ptr[17];
  for (int q = 0; q < 17; ++q) { ptr[q] = p; p += dsmc::align256(sizes[q]); }
  dsmc_step_buffers_t& b = c->rb;
  b.n = n_max; b.n_cells = n_cells; b.capacity = capacity;
  b.cell_id = (int32_t*)ptr[0]; b.vx = (double*)ptr[1]; b.vy = (double*)ptr[2]; b.vz = (double*)ptr[3];
  b.perm = (int32_t*)ptr[4]; b.cell_start = (int32_t*)ptr[5];
  b.svx = (double*)ptr[6]; b.svy = (double*)ptr[7]; b.svz = (double*)ptr[8];
  b.mom = (double*)ptr[9]; b.sigma_g_max = (double*)ptr[10]; b.pairs = (int32_t*)ptr[11];
  b.round_offsets = (int32_t*)ptr[12]; b.info = (dsmc_select_info_t*)ptr[13];
  c->r_T = (double*)ptr[14];
  b.ws = ptr[15]; b.ws_bytes = wsb;
  b.deps = (uint32_t*)ptr[16];
  c->r_n = n_max; c->r_cells = n_cells; c->r_cap = capacity; c->r_sg_ready = false;
  return DSMC_OK;
}

int dsmc_step_host(dsmc_ctx_t* c, const dsmc_gas_t* gas, const dsmc_path_t* path, int32_t n,
                   const int32_t* cell_id_h, const double* vx_h, const double* vy_h,
                   const double* vz_h, const double* T_cell_h, uint64_t step, int32_t* perm_h,
                   double* svx_h, double* svy_h, double* svz_h, int64_t* n_pairs_h,
                   void* stream) {
  CHECK_CTX(c);
  REQUIRE(c, c->r_mem, "step_host: call dsmc_ctx_reserve first");
  REQUIRE(c, n >= 0 && n <= c->r_n, "step_host: n exceeds the reserved size");
  REQUIRE(c, n == 0 || (cell_id_h && vx_h && vy_h && vz_h && svx_h && svy_h && svz_h),
          "step_host: null host array");
  if (int rc = check_gas(c, gas)) return rc;
  cudaStream_t s = S(stream);
  dsmc_step_buffers_t b = c->rb;
  b.n = n;
  const size_t n4 = 4 * (size_t)n, n8 = 8 * (size_t)n;
  if (!c->r_side) {
    if (cudaStreamCreateWithFlags(&c->r_side, cudaStreamNonBlocking) != cudaSuccess)
      return dsmc::record(c, DSMC_ERR_CUDA, "step_host: side stream");
    for (cudaEvent_t& e : c->r_ev)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
        return dsmc::record(c, DSMC_ERR_CUDA, "step_host: event");
  }
  cudaStream_t s2 = c->r_side;
  // Copies overlap the step: the cell ids upload first (alone on the host
  // link), then the velocities on the side stream while the radix passes sort
  // the cell ids, each component gathered as soon as it has landed; perm
  // downloads while the pairs are selected and updated.
  bool ok = cudaMemcpyAsync((void*)b.cell_id, cell_id_h, n4, cudaMemcpyHostToDevice, s) == cudaSuccess &&
            cudaEventRecord(c->r_ev[0], s) == cudaSuccess && cudaStreamWaitEvent(s2, c->r_ev[0], 0) == cudaSuccess &&
            cudaMemcpyAsync((void*)b.vx, vx_h, n8, cudaMemcpyHostToDevice, s2) == cudaSuccess &&
            cudaEventRecord(c->r_ev[4], s2) == cudaSuccess &&
            cudaMemcpyAsync((void*)b.vy, vy_h, n8, cudaMemcpyHostToDevice, s2) == cudaSuccess &&
            cudaEventRecord(c->r_ev[5], s2) == cudaSuccess &&
            cudaMemcpyAsync((void*)b.vz, vz_h, n8, cudaMemcpyHostToDevice, s2) == cudaSuccess &&
            cudaEventRecord(c->r_ev[1], s2) == cudaSuccess;
  if (!ok) return dsmc::record(c, DSMC_ERR_CUDA, "step_host: host-to-device copy failed");
  if (!c->r_sg_ready) {
    REQUIRE(c, T_cell_h, "step_host: T_cell_host needed on the first call");
    if (cudaMemcpyAsync(c->r_T, T_cell_h, 8 * (size_t)b.n_cells, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return dsmc::record(c, DSMC_ERR_CUDA, "step_host: copy of T_cell failed");
    int rc = dsmc_sigma_g_max_init(c, gas, b.n_cells, c->r_T, 5.0, b.sigma_g_max, stream);
    if (rc) return rc;
    c->r_sg_ready = true;
  }
  int rc = dsmc::launch_sort_keys(c, n, b.n_cells, b.cell_id, b.perm, b.cell_start, b.ws, b.ws_bytes, s);
  if (rc) return rc;
  ok = cudaEventRecord(c->r_ev[2], s) == cudaSuccess && cudaStreamWaitEvent(s2, c->r_ev[2], 0) == cudaSuccess &&
       (!perm_h || cudaMemcpyAsync(perm_h, b.perm, n4, cudaMemcpyDeviceToHost, s2) == cudaSuccess) &&
       cudaEventRecord(c->r_ev[3], s2) == cudaSuccess;
  if (!ok) return dsmc::record(c, DSMC_ERR_CUDA, "step_host: stream ordering failed");
  const double* vin[3] = {b.vx, b.vy, b.vz};
  double* vout[3] = {b.svx, b.svy, b.svz};
  const int landed[3] = {4, 5, 1};   // the event after each component's upload
  for (int q = 0; q < 3 && !rc; ++q)
    rc = cudaStreamWaitEvent(s, c->r_ev[landed[q]], 0) != cudaSuccess
             ? dsmc::record(c, DSMC_ERR_CUDA, "step_host: stream ordering failed")
             : dsmc::launch_gather_one(c, n, b.n_cells, b.cell_start, b.perm, vin[q], vout[q], s);
  if (!rc) rc = step_after_sort(c, gas, path, &b, step, stream);
  // the side stream's copies join the caller's stream whatever happened
  const bool joined = cudaStreamWaitEvent(s, c->r_ev[3], 0) == cudaSuccess;
  if (rc) return rc;
  if (!joined) return dsmc::record(c, DSMC_ERR_CUDA, "step_host: stream ordering failed");
  ok = cudaMemcpyAsync(svx_h, b.svx, n8, cudaMemcpyDeviceToHost, s) == cudaSuccess &&
       cudaMemcpyAsync(svy_h, b.svy, n8, cudaMemcpyDeviceToHost, s) == cudaSuccess &&
       cudaMemcpyAsync(svz_h, b.svz, n8, cudaMemcpyDeviceToHost, s) == cudaSuccess &&
       cudaMemcpyAsync(c->r_host_info, b.info, sizeof(dsmc_select_info_t), cudaMemcpyDeviceToHost, s) ==
           cudaSuccess;
  if (!ok) return dsmc::record(c, DSMC_ERR_CUDA, "step_host: device-to-host copy failed");
  rc = dsmc_ctx_sync_status(c, stream);
  if (n_pairs_h) *n_pairs_h = ((dsmc_select_info_t*)c->r_host_info)->n_pairs;
  return rc;
}

/* ---------------------------------------------------------------- launch shapes */

int dsmc_tune_set(dsmc_ctx_t* c, int32_t kernel, int32_t threads, int32_t blocks_per_sm) {
  CHECK_CTX(c);
  REQUIRE(c, kernel >= 0 && kernel < DSMC_TUNE_KERNELS, "tune_set: unknown kernel");
  if (threads == 0 && blocks_per_sm == 0) {
    c->tune_threads[kernel] = 0;
    c->tune_bps[kernel] = 0;
    return DSMC_OK;
  }
  REQUIRE(c, threads >= 32 && threads % 32 == 0 && threads <= dsmc::shape_info(kernel).max_threads,
          "tune_set: block size must be a multiple of 32 within the kernel's limit");
  REQUIRE(c, blocks_per_sm >= 1 && blocks_per_sm <= 64, "tune_set: blocks per SM must be 1..64");
  REQUIRE(c, (kernel != DSMC_TUNE_MOMENTS && kernel != DSMC_TUNE_MOMENT_MATCH) || threads == 256,
          "tune_set: the cell kernels run 256-thread blocks");
  c->tune_threads[kernel] = threads;
  c->tune_bps[kernel] = blocks_per_sm;
  return DSMC_OK;
}

int dsmc_tune_get(dsmc_ctx_t* c, int32_t kernel, int32_t* threads, int32_t* blocks_per_sm) {
  CHECK_CTX(c);
  REQUIRE(c, kernel >= 0 && kernel < DSMC_TUNE_KERNELS && threads && blocks_per_sm, "tune_get: bad argument");
  const dsmc::Shape s = dsmc::shape_or_default(c, kernel);
  *threads = s.threads;
  *blocks_per_sm = s.blocks_per_sm;
  return DSMC_OK;
}

int dsmc_tune_candidates(dsmc_ctx_t* c, int32_t kernel, dsmc_tune_entry_t* out, int32_t cap, int32_t* n) {
  CHECK_CTX(c);
  REQUIRE(c, kernel >= 0 && kernel < DSMC_TUNE_KERNELS && n && cap >= 0 && (cap == 0 || out),
          "tune_candidates: bad argument");
  if (cudaSetDevice(c->device) != cudaSuccess) return DSMC_ERR_CUDA;
  *n = dsmc::tune_candidates(kernel, out, cap);
  return DSMC_OK;
}

}  // extern "C"

namespace {

// Time every candidate shape of `kernel` with `launch` (one untimed launch,
// then `reps` between events), keep the fastest; entries go to trials.
template <class F>
int tune_kernel(dsmc_ctx* c, int kernel, int reps, cudaStream_t s, F&& launch, dsmc_tune_entry_t* trials,
                int cap, int* nt) {
  dsmc_tune_entry_t cand[64];
  const int nc = dsmc::tune_candidates(kernel, cand, 64);
  if (nc < 1) return DSMC_OK;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return dsmc::record(c, DSMC_ERR_CUDA, "autotune: event");
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return dsmc::record(c, DSMC_ERR_CUDA, "autotune: event"); }
  const int t0 = c->tune_threads[kernel], b0 = c->tune_bps[kernel];
  int best = -1, rc = DSMC_OK;
  for (int q = 0; q < nc && q < 64; ++q) {
    c->tune_threads[kernel] = cand[q].threads;
    c->tune_bps[kernel] = cand[q].blocks_per_sm;
    rc = launch();
    if (!rc && cudaEventRecord(e0, s) != cudaSuccess) rc = DSMC_ERR_CUDA;
    for (int r = 0; r < reps && !rc; ++r) rc = launch();
    if (!rc && cudaEventRecord(e1, s) != cudaSuccess) rc = DSMC_ERR_CUDA;
    if (!rc) rc = dsmc_ctx_sync_status(c, s);
    if (rc) break;
    float el = 0.f;
    cudaEventElapsedTime(&el, e0, e1);
    cand[q].ms = el / (float)reps;
    if (trials && *nt < cap) trials[*nt] = cand[q];
    ++*nt;
    if (best < 0 || cand[q].ms < cand[best].ms) best = q;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc || best < 0) {
    c->tune_threads[kernel] = t0;
    c->tune_bps[kernel] = b0;
    return rc;
  }
  c->tune_threads[kernel] = cand[best].threads;
  c->tune_bps[kernel] = cand[best].blocks_per_sm;
  return DSMC_OK;
}

}  // namespace

extern "C" {

int dsmc_autotune_step(dsmc_ctx_t* c, const dsmc_gas_t* gas, const dsmc_path_t* path,
                       const dsmc_step_buffers_t* B, uint64_t step, int32_t reps,
                       dsmc_tune_entry_t* trials, int32_t cap, int32_t* n_trials, void* stream) {
  CHECK_CTX(c);
  REQUIRE(c, gas && path && B && n_trials && reps >= 1 && cap >= 0, "autotune_step: bad argument");
  REQUIRE(c, !c->capturing, "autotune_step: not during a graph capture");
  *n_trials = 0;
  cudaStream_t s = S(stream);
  int rc = dsmc_step(c, gas, path, B, step, stream);
  if (!rc) rc = dsmc_ctx_sync_status(c, stream);
  if (rc) return rc;
  if (B->n == 0 || B->n_cells == 0) return DSMC_OK;
  int nt = 0;
  rc = tune_kernel(c, DSMC_TUNE_GATHER, reps, s, [&] {
    return dsmc::launch_gather(c, B->n, B->n_cells, B->cell_start, B->perm, B->vx, B->vy, B->vz, B->svx,
                               B->svy, B->svz, s);
  }, trials, cap, &nt);
  if (!rc) rc = tune_kernel(c, DSMC_TUNE_MOMENTS, reps, s, [&] {
    return dsmc::launch_moments(c, B->n_cells, B->cell_start, B->svx, B->svy, B->svz, B->mom, s);
  }, trials, cap, &nt);
  if (!rc && path->path == DSMC_PATH_VHS)
    rc = tune_kernel(c, DSMC_TUNE_COLLIDE_VHS, reps, s, [&] {
      return dsmc_collide_vhs(c, gas, step, B->n, B->pairs, B->deps, B->round_offsets, B->info, B->svx, B->svy,
                              B->svz, B->ws, B->ws_bytes, stream);
    }, trials, cap, &nt);
  if (!rc && path->path == DSMC_PATH_TABLE)
    rc = tune_kernel(c, DSMC_TUNE_COLLIDE_TABLE, reps, s, [&] {
      return dsmc_collide_table(c, gas, path->table, step, B->n, B->pairs, B->deps, B->round_offsets, B->info,
                                B->svx, B->svy, B->svz, nullptr, B->ws, B->ws_bytes, stream);
    }, trials, cap, &nt);
  if (!rc && path->path == DSMC_PATH_JAGER)
    rc = tune_kernel(c, DSMC_TUNE_COLLIDE_JAGER, reps, s, [&] {
      return dsmc_collide_jager(c, gas, path->pot, path->n_nodes, step, B->n, B->pairs, B->deps, B->round_offsets,
                                B->info, B->svx, B->svy, B->svz, nullptr, B->ws, B->ws_bytes, stream);
    }, trials, cap, &nt);
  if (!rc) rc = tune_kernel(c, DSMC_TUNE_MOMENT_MATCH, reps, s, [&] {
    return dsmc::launch_moment_match(c, B->n_cells, B->cell_start, B->mom, B->svx, B->svy, B->svz, s);
  }, trials, cap, &nt);
  *n_trials = nt;
  return rc;
}

int dsmc_autotune_chi(dsmc_ctx_t* c, const dsmc_gas_t* gas, const dsmc_potential_t* pot, int32_t n_nodes,
                      int64_t n, const float* b, const float* g, float* chi, int32_t reps,
                      dsmc_tune_entry_t* trials, int32_t cap, int32_t* n_trials, void* stream) {
  CHECK_CTX(c);
  REQUIRE(c, n_trials && reps >= 1 && cap >= 0, "autotune_chi: bad argument");
  *n_trials = 0;
  if (n == 0) return DSMC_OK;
  int nt = 0;
  const int rc = tune_kernel(c, DSMC_TUNE_JAGER_CHI, reps, S(stream), [&] {
    return dsmc_jager_chi(c, gas, pot, n_nodes, n, b, g, chi, stream);
  }, trials, cap, &nt);
  *n_trials = nt;
  return rc;
}

}  // extern "C"
