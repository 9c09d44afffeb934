/*
 * dsmc.h -- C ABI of the GB300 (sm_103a) DSMC collision-step library.
 *
 * Implements the collision step of "Physics Constrained Neural Collision
 * Operators for VHS Surrogates and Ab Initio Angle Prediction in DSMC"
 * (arXiv 2602.21244): cell sort, No-Time-Counter pair selection, one of three
 * pair-update rules (VHS isotropic scatter, Jager-potential deflection angle,
 * neural collision operator) and cell-wise moment matching, plus the
 * training step of the neural operator.
 *
 * Conventions (every entry point):
 *  - Pointers are DEVICE pointers owned by the caller, unless the name of
 *    the argument ends in _host.  The library never frees or keeps them.
 *  - Calls are asynchronous on the given stream (a cudaStream_t passed as
 *    void*; NULL = the legacy default stream).  The return value reports
 *    argument and launch errors only.  Errors found on the device
 *    (capacity overflow, a bounded wait that ran out, non-finite input)
 *    are recorded in the context's status word; dsmc_ctx_sync_status()
 *    waits for the stream and returns (and clears) that word.
 *  - Velocities are double precision, structure of arrays (vx, vy, vz),
 *    in m/s.  Particle and cell indices are int32 (N < 2^31).
 *  - Scratch memory is a caller-provided workspace of the size returned by
 *    the matching *_workspace_size() query, 256-byte aligned.
 *  - Results depend only on the inputs, the seed and the step index, never
 *    on the launch configuration.
 *  - Status codes: 0 = DSMC_OK, negative = error (see below).
 *  - The collide kernels of one context share its grid-barrier words: direct
 *    collide calls of one context must not overlap on the GPU (issue them on
 *    one stream, or use one context per stream).  A captured step graph has
 *    words of its own and may overlap direct calls.
 */
#ifndef DSMC_H_
#define DSMC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DSMC_ABI_VERSION 3

enum {
  DSMC_OK = 0,
  DSMC_ERR_ARG = -1,         /* bad argument (null pointer, size, cell id out of range) */
  DSMC_ERR_CUDA = -2,        /* a CUDA runtime call failed */
  DSMC_ERR_CAPACITY = -3,    /* more accepted pairs than the pair buffer holds */
  DSMC_ERR_TIMEOUT = -4,     /* a bounded device-side wait ran out */
  DSMC_ERR_NONFINITE = -5,   /* NaN or Inf in an input velocity */
  DSMC_ERR_UNSUPPORTED = -6  /* shape outside what the kernels handle */
};

/* Update rules of the collision step (Sec. 2.1: only the scattering rule changes). */
enum { DSMC_PATH_VHS = 0, DSMC_PATH_JAGER = 1, DSMC_PATH_NEURAL = 2, DSMC_PATH_TABLE = 3 };

/* Largest number of conflict-free rounds one step may need (see dsmc_select_pairs). */
#define DSMC_MAX_ROUNDS 1024

/* Bucket order of the selection's pair list (dsmc_select_pairs_ordered). */
enum { DSMC_ORDER_ROUNDS = 0, DSMC_ORDER_LEVELS = 1 };

typedef struct dsmc_ctx dsmc_ctx_t;

/* Gas and selection parameters (Sec. 2.2).
 *  model 0: Bird's VHS cross section
 *           sigma(g) = pi d_ref^2 (2 k T_ref/(m_r g^2))^(omega-1/2) / Gamma(5/2-omega),
 *           m_r = mass/2 (omega = 1/2 is the hard sphere);
 *  model 1: constant sigma = pi b_max^2 (impact-parameter cut-off of the
 *           ab-initio paths, Sec. 3.4.2: b <= b_max).
 *  fn_over_vc = F_N / V_c, the number of real molecules per simulator
 *  particle divided by the cell volume (1/m^3). */
typedef struct {
  double mass;       /* kg */
  double d_ref;      /* m */
  double omega;
  double T_ref;      /* K */
  double fn_over_vc; /* 1/m^3 */
  double dt;         /* s */
  uint64_t seed;     /* Philox key */
  int32_t model;
  int32_t pad_;
  double b_max;      /* m */
} dsmc_gas_t;

/* Interaction potential for the deflection angle (Sec. 3.4.1), r in
 * Angstrom, V/k_B in Kelvin.
 *  kind 0: Jager form, Eq. (jager_potential) with Tang-Toennies damping
 *          Eq. (damping) for r >= 0.4 R_eps, screened Coulomb
 *          At exp(-at r)/r below;
 *  kind 1: hard sphere of diameter d_hs (closed-form check);
 *  kind 2: inverse power kappa / r^p. */
typedef struct {
  int32_t kind;
  int32_t pad_;
  double A, a1, a2, am1, am2; /* repulsion A exp(a1 r + a2 r^2 + am1/r + am2/r^2) */
  double beta;                /* damping constant (the paper's "b" in f_n(b r)) */
  double C[6];                /* C6, C8, C10, C12, C14, C16 */
  double R_eps;
  double At, at;
  double d_hs;
  double kappa, p;
} dsmc_potential_t;

/* Neural collision operator (Sec. 2.2 Eq. mlp_input / mlp_output).
 *  d_in 8: x = [v_r/sigma_v (3), T_cell/T_ref (1), xi (4)];
 *  d_in 6: x = [v_r/sigma_v (3), xi (3)] (the paper's 6-input form).
 *  n_hidden hidden layers of `width` units (the tensor-core path takes
 *  width 128 and 1..4 hidden layers), act 0 = SiLU, 1 = ReLU, then a
 *  linear layer to d_out = 3. */
typedef struct {
  int32_t d_in, width, n_hidden, d_out, act, pad_;
  double sigma_v; /* m/s */
  double T_ref;   /* K */
  double eps;     /* projection safeguard on ||y|| (normalised units) */
} dsmc_mlp_t;

/* Deflection-angle table of the look-up path (Sec. 3.4.4): chi[j nb + i] =
 * chi(b_max i/(nb-1), exp(lnE_min + j (lnE_max - lnE_min)/(nE-1))), i.e. a
 * uniform grid in b/b_max over [0, 1] and in ln(E_r/k_B) over [lnE_min,
 * lnE_max], both ends included.  chi: device memory, FP32. */
typedef struct {
  const float* chi;
  int32_t nb, nE;      /* nodes along b/b_max and along ln E, each 2..4096 */
  double lnE_min, lnE_max;
} dsmc_chi_table_t;

/* Written by dsmc_select_pairs (device memory). */
typedef struct {
  int64_t n_pairs;      /* accepted pairs this step */
  int64_t n_candidates; /* NTC candidates drawn this step */
  int32_t n_rounds;     /* conflict-free rounds */
  int32_t pad_;
} dsmc_select_info_t;

/* ---------------------------------------------------------------- context */

/* Create a context on `device` (allocates the status word and small
 * per-device tables; the only allocation the library makes besides
 * dsmc_ctx_reserve).  Returns DSMC_ERR_CUDA if the device is unusable. */
int dsmc_ctx_create(dsmc_ctx_t** ctx, int device);
void dsmc_ctx_destroy(dsmc_ctx_t* ctx);
/* Wait for `stream`, return the first device-side error since the last
 * call (DSMC_OK if none) and clear it. */
int dsmc_ctx_sync_status(dsmc_ctx_t* ctx, void* stream);
/* Text of the last host-side error of this context (static storage). */
const char* dsmc_last_error(dsmc_ctx_t* ctx);
int dsmc_abi_version(void);
/* Number of CUDA kernels this context has launched so far (for reporting). */
int64_t dsmc_ctx_launch_count(dsmc_ctx_t* ctx);

/* ---------------------------------------------------------------- sort */

/* Sec. 2.6 (1): sort particles by cell index so each cell's particles are
 * contiguous.  Stable counting sort: perm[s] is the input index of sorted
 * slot s, slots of a cell keep the input order.  cell_start[n_cells+1]
 * holds each cell's first slot; s{x,y,z} receive the gathered velocities
 * (s{x,y,z} must not overlap v{x,y,z}).  cell_id[i] outside
 * [0, n_cells) records DSMC_ERR_ARG; such a particle belongs to no cell, and
 * the entries of perm and s{x,y,z} past cell_start[n_cells] are unspecified. */
size_t dsmc_sort_workspace_size(int32_t n, int32_t n_cells);
int dsmc_sort_cells(dsmc_ctx_t* ctx, int32_t n, int32_t n_cells, const int32_t* cell_id,
                    const double* vx, const double* vy, const double* vz, int32_t* perm,
                    int32_t* cell_start, double* svx, double* svy, double* svz, void* ws,
                    size_t ws_bytes, void* stream);

/* Allocation-free variant of dsmc_sort_cells; the paper has no counterpart.
 * For callers that cannot allocate device memory at the point of the call:
 * a solver that reserved all of the GPU's memory for its particle arrays up
 * front, code that runs where cudaMalloc is not allowed or would stall the
 * device (it can synchronise), or a host that hands the library only the
 * arrays it owns.  It needs no context and no workspace: its scratch is one
 * file-scope device array of about 5.2 MB that every GPU loading this
 * library holds until the process exits, so it sorts at most
 * DSMC_STATIC_SORT_MAX_N particles into at most DSMC_STATIC_SORT_MAX_CELLS
 * cells and returns DSMC_ERR_UNSUPPORTED for anything larger.
 *  - Arguments and results as dsmc_sort_cells (device pointers, caller-owned;
 *    same stable order, bit for bit).  `status` (optional device int, may be
 *    NULL) receives DSMC_ERR_ARG if a cell id is out of range; it must be
 *    zeroed by the caller beforehand.
 *  - The call makes no cudaMalloc/cudaFree and calls no allocating library
 *    routine.  Its first call on a device looks up the scratch array's
 *    device address with that device current (cudaGetSymbolAddress); make
 *    that first call before any stream capture.
 *  - Every call shares the one array: calls that overlap on the GPU (two
 *    streams, two host threads) race and corrupt each other's result.
 *    Serialise them on one stream. */
#define DSMC_STATIC_SORT_MAX_N (1 << 20)
#define DSMC_STATIC_SORT_MAX_CELLS (1 << 18)
int dsmc_sort_cells_static(int32_t n, int32_t n_cells, const int32_t* cell_id, const double* vx,
                           const double* vy, const double* vz, int32_t* perm, int32_t* cell_start,
                           double* svx, double* svy, double* svz, int* status, void* stream);

/* Per-cell moments of sorted velocities:
 * mom[5k..5k+4] = {N, sum vx, sum vy, sum vz, Theta = sum |v - u|^2},
 * u = sum v / N, as exact integer sums: each component is rounded to the
 * cell's unit (the unit in the last place of its largest component, 2^c
 * coarser for cells of 2^(9+c) particles or more so that the sums fit 64
 * bits), the sums and the centred sum of squares are exact (128-bit), and
 * only the results are converted to FP64 (independent of the order of the
 * sums).  Non-finite velocities record DSMC_ERR_NONFINITE. */
int dsmc_cell_moments(dsmc_ctx_t* ctx, int32_t n_cells, const int32_t* cell_start,
                      const double* vx, const double* vy, const double* vz, double* mom,
                      void* stream);

/* ---------------------------------------------------------------- selection */

/* Initial (sigma g)_max of each cell: sigma(g0) g0, g0 = factor sqrt(2 k T_cell/m). */
int dsmc_sigma_g_max_init(dsmc_ctx_t* ctx, const dsmc_gas_t* gas, int32_t n_cells,
                          const double* T_cell, double factor, double* sigma_g_max,
                          void* stream);

/* Sec. 2.2: NTC pair selection over cell-sorted particles.
 *  Cell k with N >= 2 draws M = floor(1/2 N(N-1) (F_N/V_c) (sigma g)_max dt + U)
 *  candidates (Philox tag 1); candidate m picks i, j != i uniformly (tag 2)
 *  and is accepted iff U' < sigma(g) g / (sigma g)_max with g from the
 *  velocities as passed in (the pre-step state).  (sigma g)_max is raised
 *  afterwards to the largest sigma g among the cell's candidates.
 *  Accepted pairs act in candidate order; round(p) = 1 + max(last round of
 *  i, last round of j) splits them into rounds of disjoint pairs that,
 *  applied in round order, reproduce the sequential result exactly.
 *  Output: pairs[4p..4p+3] = {i, j, cell, m} (sorted slot indices, cell,
 *  candidate index) grouped by round (inside a round in cell order, and in
 *  candidate order within a cell),
 *  deps[p] = (1-based round of the previous pair of particle i) | (that of
 *  j) << 16, 0 = none (the collide kernels order their work by it),
 *  round_offsets[r] = first pair of round r (the array holds
 *  DSMC_MAX_ROUNDS + 1 entries; r = 0..n_rounds are meaningful), *info.
 *  More than `capacity` pairs records DSMC_ERR_CAPACITY and writes none;
 *  more than DSMC_MAX_ROUNDS rounds records DSMC_ERR_UNSUPPORTED. */
size_t dsmc_select_workspace_size(int32_t n, int32_t n_cells, int64_t capacity);
int dsmc_select_pairs(dsmc_ctx_t* ctx, const dsmc_gas_t* gas, int32_t n, int32_t n_cells,
                      const int32_t* cell_start, const double* vx, const double* vy,
                      const double* vz, double* sigma_g_max, uint64_t step, int64_t capacity,
                      int32_t* pairs, uint32_t* deps, int32_t* round_offsets, dsmc_select_info_t* info,
                      void* ws, size_t ws_bytes, void* stream);
/* dsmc_select_pairs with the pair list's buckets chosen by `order`:
 * DSMC_ORDER_ROUNDS is dsmc_select_pairs.  DSMC_ORDER_LEVELS buckets the
 * same pairs by claim level = round + (n_rounds - 1 - the last round of the
 * pair's cell): every pair of a cell moves by the same amount, so each
 * particle's pairs keep their order and the levels are again conflict-free
 * buckets that reproduce the sequential result in level order, but a cell
 * with few rounds is deferred to the end of the list while the cells with
 * the longest dependency chains start at once.  round_offsets[l] = first
 * pair of level l (l = 0..n_rounds), inside a level in cell order and
 * candidate order within a cell; deps[p] holds the 1-based levels of the
 * previous pairs of i and j (0 = none); *info (n_rounds included) is as for
 * rounds.  The collide calls take either list.  Another order returns
 * DSMC_ERR_ARG. */
int dsmc_select_pairs_ordered(dsmc_ctx_t* ctx, const dsmc_gas_t* gas, int32_t n, int32_t n_cells,
                              const int32_t* cell_start, const double* vx, const double* vy,
                              const double* vz, double* sigma_g_max, uint64_t step, int64_t capacity,
                              int32_t* pairs, uint32_t* deps, int32_t* round_offsets, dsmc_select_info_t* info,
                              int32_t order, void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------- pair updates */

/* Common to the three collide calls: n particles (the sorted slots the
 * pairs index), pairs / deps / round_offsets / info from dsmc_select_pairs.
 * The kernels apply the pairs in round order without grid-wide barriers: a
 * pair waits (bounded; DSMC_ERR_TIMEOUT if it runs out) until the previous
 * pairs of its two particles are done, which gives the result of applying
 * the rounds one after another.  ws: dsmc_collide_workspace_size(n) bytes
 * of scratch (one done stamp per particle, cleared by each call). */
size_t dsmc_collide_workspace_size(int32_t n);

/* VHS isotropic scatter (the phenomenological kernel the paper replaces,
 * Sec. 2.1) with the centre-of-mass update of Sec. 2.3:
 *  cos chi = 2U1 - 1, eps = 2 pi U2 (Philox tag 3, counter = candidate m),
 *  v_r' = |v_r| (cos chi, sin chi cos eps, sin chi sin eps),
 *  v_i = v_cm + v_r'/2, v_j = v_cm - v_r'/2; in place. */
int dsmc_collide_vhs(dsmc_ctx_t* ctx, const dsmc_gas_t* gas, uint64_t step, int32_t n,
                     const int32_t* pairs, const uint32_t* deps, const int32_t* round_offsets,
                     const dsmc_select_info_t* info, double* vx, double* vy, double* vz,
                     void* ws, size_t ws_bytes, void* stream);

/* Sec. 3.4.2 / 3.4.4: deflection angle of the classical scattering integral
 *  chi(b, E) = pi - 2 b int_{r_min}^inf dr / (r^2 sqrt(1 - b^2/r^2 - V(r)/E)),
 *  E = E_r/k_B = m g^2/(4 k_B), r_min the largest root of the radicand.
 *  FP32 bracket and quadrature (u = r_min/r, u = 1 - s^2, n_nodes-point
 *  Gauss-Legendre in s, n_nodes in [8, 128]; min(4 n_nodes, 128) points for
 *  energies below 1.5 well depths of the Jager form, where near-orbiting
 *  pairs make the integrand steep) with an FP64 Halley refinement of r_min.  Signed: attraction gives chi < 0.
 *  b in Angstrom, g in m/s, n pairs. */
int dsmc_jager_chi(dsmc_ctx_t* ctx, const dsmc_gas_t* gas, const dsmc_potential_t* pot,
                   int32_t n_nodes, int64_t n, const float* b, const float* g, float* chi,
                   void* stream);

/* Pair update with the deflection angle: b = b_max sqrt(U1), eps = 2 pi U2
 *  (tag 4); v_r' = cos chi v_r + |v_r| sin chi (cos eps c + sin eps a) with
 *  c = (0, v_z, -v_y)/q, a = (q^2, -v_x v_y, -v_x v_z)/(|v_r| q),
 *  q = sqrt(v_y^2 + v_z^2) (Bird 1994, Eq. 2.22; for q = 0, c = (0,1,0) and
 *  a = c x v_r/|v_r|).  chi_out (optional, may be NULL) receives each
 *  pair's chi in pair order. */
int dsmc_collide_jager(dsmc_ctx_t* ctx, const dsmc_gas_t* gas, const dsmc_potential_t* pot,
                       int32_t n_nodes, uint64_t step, int32_t n, const int32_t* pairs,
                       const uint32_t* deps, const int32_t* round_offsets, const dsmc_select_info_t* info,
                       double* vx, double* vy, double* vz, float* chi_out, void* ws, size_t ws_bytes,
                       void* stream);

/* Macroscopic validation (Eq. chapman_enskog and the two integrals after
 * it), reading R8.  Transport cross-section
 *   Q2(E) = 2 pi int_0^{b_max} (1 - cos^2 chi(b, E)) b db
 *         = pi b_max^2 int_0^1 sin^2 chi(b_max sqrt(u), E) du
 * by a composite 16-point Gauss-Legendre rule (b_panels equal panels of
 * [0, 1] in u = (b/b_max)^2), chi at every node as in dsmc_jager_chi.
 * E_kelvin: n_E energies E_r/k_B > 0 (K), device memory; b_max_A in Angstrom;
 * q2: n_E values in m^2, device memory.  An energy that is not positive and
 * finite records DSMC_ERR_ARG on the device.  Deterministic. */
int dsmc_transport_q2(dsmc_ctx_t* ctx, const dsmc_potential_t* pot, int32_t n_nodes, int32_t n_E,
                      const double* E_kelvin, double b_max_A, int32_t b_panels, double* q2, void* stream);
/* Collision integral and first-order Chapman-Enskog viscosity at n_T
 * temperatures (device memory, K):
 *   Omega22(T) = 1/(4 (kT)^4) int_0^inf E^3 Q2(E) exp(-E/kT) dE
 *              = 1/4 int_0^60 x^3 e^-x Q2(x kT) dx   (x_panels 16-point panels),
 *   mu(T) = 5/16 sqrt(pi m k T) / Omega22(T),  m = gas->mass.
 * omega22 (m^2) and mu (Pa s): n_T values each, device memory.  ws: caller
 * workspace of dsmc_transport_workspace_size(n_T, x_panels) bytes (Q2 at the
 * n_T x 16 x_panels energies of the rule). */
size_t dsmc_transport_workspace_size(int32_t n_T, int32_t x_panels);
int dsmc_transport_viscosity(dsmc_ctx_t* ctx, const dsmc_gas_t* gas, const dsmc_potential_t* pot, int32_t n_nodes,
                             int32_t n_T, const double* T_kelvin, double b_max_A, int32_t b_panels,
                             int32_t x_panels, double* omega22, double* mu, void* ws, size_t ws_bytes,
                             void* stream);

/* chi-MLP surrogate (Sec. 3.4, Fig. nn_architecture; reading R9): inputs
 * x = [ln(E_r)*, b/b_max] with ln(E_r)* = (ln(E_r/k_B) - ln 5)/(ln 60000 - ln 5),
 * hidden layers 512, 512, 512, 256, 128 with SiLU, one Softplus output
 * y ~ ln(1 + chi), chi = e^y - 1.  Weights: bf16 bits, layers row-major
 * [out x in] concatenated (512x2, 512x512, 512x512, 256x512, 128x256, 1x128);
 * bias: FP32, concatenated (1921 values).  On the tensor cores with the input
 * as two bf16 terms and hidden activations 1-4 as single bf16 terms, FP32
 * accumulation; the output layer an FP32 dot product.
 *
 * dsmc_chi_mlp_pack writes the weights once into `packed` (device memory of
 * dsmc_chi_mlp_packed_size() bytes, 16-byte aligned) in the operand layout
 * the kernel streams.  dsmc_chi_mlp_forward: n rows x [2] (FP32, device) ->
 * y (Softplus output) and/or chi (e^y - 1), either may be NULL.
 * dsmc_chi_mlp_table: the nE x nb table of Sec. 3.4.4 (row j: ln(E_r)* =
 * j/(nE-1); column i: b/b_max = i/(nb-1)), chi = e^y - 1, FP32 device memory. */
size_t dsmc_chi_mlp_packed_size(void);
int dsmc_chi_mlp_pack(dsmc_ctx_t* ctx, const uint16_t* w_bits, void* packed, void* stream);
int dsmc_chi_mlp_forward(dsmc_ctx_t* ctx, const void* packed, const float* bias, int64_t n, const float* x,
                         float* y, float* chi, void* stream);
int dsmc_chi_mlp_table(dsmc_ctx_t* ctx, const void* packed, const float* bias, int32_t nb, int32_t nE,
                       float* table, void* stream);

/* Sec. 3.4.4: fill a chi table with the exact deflection angle (the
 * computation of dsmc_jager_chi at every node; b_max from gas->b_max).
 * table: nE x nb FP32, device memory. */
int dsmc_chi_table_build(dsmc_ctx_t* ctx, const dsmc_gas_t* gas, const dsmc_potential_t* pot, int32_t n_nodes,
                         int32_t nb, int32_t nE, double lnE_min, double lnE_max, float* table, void* stream);
/* Sec. 3.4.4 look-up path: the pair update of dsmc_collide_jager with chi by
 * bilinear interpolation in `table` at (b/b_max, ln(E_r/k_B)); ln E outside
 * the table is clamped to its range.  b/b_max = sqrt(U1) and eps = 2 pi U2
 * from tag 4, as the Jager path.  chi_out (optional) as dsmc_collide_jager. */
int dsmc_collide_table(dsmc_ctx_t* ctx, const dsmc_gas_t* gas, const dsmc_chi_table_t* table, uint64_t step,
                       int32_t n, const int32_t* pairs, const uint32_t* deps, const int32_t* round_offsets,
                       const dsmc_select_info_t* info, double* vx, double* vy, double* vz, float* chi_out,
                       void* ws, size_t ws_bytes, void* stream);

/* Sec. 2.2-2.3: neural collision operator on the tcgen05 tensor cores.
 *  x as in dsmc_mlp_t (xi: Box-Muller normals from tag 5, subs 0 and 1;
 *  T_cell = m Theta_pre / (3 k_B N) from mom_pre), bf16 operands with FP32
 *  accumulation, y = f_theta(x), u = y/||y|| (isotropic direction from tag 3
 *  if ||y|| <= eps), v_r' = |v_r| u, centre-of-mass update in FP64.
 *  weights_bf16: each layer's row-major [out x in] matrix, concatenated;
 *  biases: each layer's bias (FP32), concatenated.  Requires width 128,
 *  d_out 3, d_in 6 or 8, 1..4 hidden layers.  The MLP input enters the
 *  first layer as two bf16 terms (hi + lo) sharing the first layer's weights.
 *  u_out (optional, may be NULL) receives each pair's unit direction u
 *  (FP32 [n_pairs x 3], pair order). */
int dsmc_collide_neural(dsmc_ctx_t* ctx, const dsmc_gas_t* gas, const dsmc_mlp_t* mlp,
                        const uint16_t* weights_bf16, const float* biases, uint64_t step,
                        const double* mom_pre, int32_t n, const int32_t* pairs, const uint32_t* deps,
                        const int32_t* round_offsets, const dsmc_select_info_t* info,
                        double* vx, double* vy, double* vz, float* u_out, void* ws, size_t ws_bytes,
                        void* stream);

/* The MLP alone on the tensor cores: y[n x 3] = f_theta(x[n x d_in]) with x
 * and y FP32 row-major (x rounded to bf16 on the way in), same weight
 * layout as dsmc_collide_neural. */
int dsmc_mlp_forward(dsmc_ctx_t* ctx, const dsmc_mlp_t* mlp, const uint16_t* weights_bf16,
                     const float* biases, int64_t n, const float* x, float* y, void* stream);

/* Diagnostic with no counterpart in the paper: D[128 x N] = A[128 x K] B[N x K]^T
 * (bf16 row-major in, FP32 row-major out) through the same shared-memory
 * operand layout, descriptors and tcgen05.mma issue as the MLP, on one CTA.
 * N a multiple of 16 in [16, 256], K a multiple of 16 in [16, 128].
 * layout bit 0: A held MN-major in shared memory, bit 1: B MN-major (as the
 * backward pass reads them), bit 2: exchange the two descriptor offsets of
 * MN-major operands (a check of the descriptor convention), bit 3: A in
 * tensor memory instead of shared memory (row m in lane m, two bf16 per
 * 32-bit column; not with bit 0). */
int dsmc_tc_selftest(dsmc_ctx_t* ctx, int32_t N, int32_t K, int32_t layout, const uint16_t* A,
                     const uint16_t* B, float* D, void* stream);

/* Diagnostic with no counterpart in the paper (failure detection): runs a
 * kernel whose bounded wait can never be satisfied -- which 0: a grid
 * barrier that one block never reaches; which 1: an mbarrier that no
 * tensor-core commit completes; which 2: a pair-dependency wait on a done
 * stamp that nothing sets -- so that the wait runs out after limit_ns
 * (at most 2 s) and records DSMC_ERR_TIMEOUT in the status word.  Nothing
 * traps or spins without bound; the context stays usable. */
int dsmc_selftest_timeout(dsmc_ctx_t* ctx, int32_t which, uint64_t limit_ns, void* stream);

/* Diagnostic with no counterpart in the paper (roofline denominators of
 * the arithmetic pipes): a kernel of `blocks` x `threads` threads (threads a
 * multiple of 32, at most 256), each repeating `iters` times 32 dependent
 * operations of one kind spread over 8 independent chains -- which 0: FP32
 * FMA, 1: paired FP32 FMA (fma.rn.f32x2), 2: FP64 FMA, 3: the
 * special-function unit's ex2.approx.f32 -- and writing one float per
 * thread to `sink` (device memory, blocks x threads floats) so that no work
 * is optimised away.  dsmc_selftest_peak_ops gives the operations one thread
 * performs (FLOPs for the FMA kinds, 2 per FMA and 4 per paired FMA;
 * results for ex2; -1 for bad arguments); the caller times the launch. */
/* Diagnostic with no counterpart in the paper: the FP64 helpers of the
 * turning-point refinement against CUDA's own routines, y[i] = f(x[i]) for
 * n values (device memory) -- which 0: the refinement's exponential (Cody-
 * Waite reduction by ln 2, Taylor polynomial to degree 12; |x| < 700),
 * 1: CUDA's exp, 2: the refinement's reciprocal (FP32 seed and two Newton
 * steps; x positive, inside the FP32 normal range), 3: 1.0 / x. */
int dsmc_selftest_math(dsmc_ctx_t* ctx, int32_t which, int64_t n, const double* x, double* y, void* stream);

int64_t dsmc_selftest_peak_ops(int32_t which, int32_t iters);
int dsmc_selftest_peak(dsmc_ctx_t* ctx, int32_t which, int32_t blocks, int32_t threads, int32_t iters,
                       float* sink, void* stream);

/* ---------------------------------------------------------------- moment matching */

/* Sec. 2.5, centred: per cell v <- u_pre + alpha (v - u_post),
 * alpha = sqrt(Theta_pre/Theta_post) (1 if N < 2 or Theta_post = 0), from
 * mom_pre of dsmc_cell_moments.  Restores each cell's momentum and kinetic
 * energy; equals Eq. (cell_energy_clamp) when the cell mean velocity is 0. */
int dsmc_moment_match(dsmc_ctx_t* ctx, int32_t n_cells, const int32_t* cell_start,
                      const double* mom_pre, double* vx, double* vy, double* vz,
                      void* stream);

/* ---------------------------------------------------------------- whole step */

/* Buffers of one collision step (all device memory, caller-owned).
 * Input: cell_id, vx, vy, vz (unsorted).  Output: perm, cell_start and the
 * sorted, post-collision s{x,y,z}; mom (pre moments), sigma_g_max (in/out),
 * pairs / deps / round_offsets / info as in dsmc_select_pairs (deps:
 * `capacity` uint32).  ws: dsmc_step_workspace_size bytes, shared by the
 * phases. */
typedef struct {
  int32_t n, n_cells;
  int64_t capacity;
  const int32_t* cell_id;
  const double *vx, *vy, *vz;
  int32_t* perm;
  int32_t* cell_start;
  double *svx, *svy, *svz;
  double* mom;
  double* sigma_g_max;
  int32_t* pairs;
  int32_t* round_offsets;
  dsmc_select_info_t* info;
  void* ws;
  size_t ws_bytes;
  uint32_t* deps;
} dsmc_step_buffers_t;

/* Path-specific parameters of a step (unused fields may be NULL/0). */
typedef struct {
  int32_t path;    /* DSMC_PATH_* */
  int32_t n_nodes; /* Jager quadrature nodes */
  const dsmc_potential_t* pot;
  const dsmc_mlp_t* mlp;
  const uint16_t* weights_bf16;
  const float* biases;
  const dsmc_chi_table_t* table; /* DSMC_PATH_TABLE */
} dsmc_path_t;

size_t dsmc_step_workspace_size(int32_t n, int32_t n_cells, int64_t capacity);
/* One collision step: sort, pre moments, selection, pair updates of the
 * chosen path, moment matching (Sec. 2.1-2.6).  The pair list in `buf` is
 * bucketed by claim level (DSMC_ORDER_LEVELS) on DSMC_PATH_NEURAL and by
 * round on the other paths. */
int dsmc_step(dsmc_ctx_t* ctx, const dsmc_gas_t* gas, const dsmc_path_t* path,
              const dsmc_step_buffers_t* buf, uint64_t step, void* stream);

/* The same step fused into one pass (Sec. 2.2-2.5): after the cell sort's
 * keys, one persistent kernel stages groups of consecutive cells in shared
 * memory once and runs their gather, pre moments, NTC selection, rounds,
 * pair updates and moment matching there, so each particle's velocity is
 * read from and written to device memory once.  Paths: DSMC_PATH_VHS and
 * DSMC_PATH_TABLE (others return DSMC_ERR_UNSUPPORTED).  Same buffers and
 * results as dsmc_step -- bit for bit: perm, cell_start, s{x,y,z}, mom,
 * sigma_g_max and *info (n_pairs, n_candidates, n_rounds) -- except that no
 * pair list is produced: `pairs`, `deps` and `round_offsets` are left
 * unspecified.  A cell whose particles or candidates exceed a shared-memory
 * batch (1024 particles, 3072 candidates) takes 12 bytes of scratch per
 * candidate from `pairs` (capacity entries); if that runs out,
 * DSMC_ERR_CAPACITY is recorded and the cell is not collided; a cell of more
 * than 65536 particles records DSMC_ERR_UNSUPPORTED the same way.  ws:
 * dsmc_step_workspace_size bytes.  Not captured by dsmc_step_graph_capture. */
int dsmc_step_fused(dsmc_ctx_t* ctx, const dsmc_gas_t* gas, const dsmc_path_t* path,
                    const dsmc_step_buffers_t* buf, uint64_t step, void* stream);

/* Capture one whole step -- dsmc_step with these arguments -- as a CUDA
 * graph owned by the context (replacing any earlier one).  The buffers must
 * stay allocated while the graph is used.  `stream` must be a non-default
 * stream; nothing runs during the capture.  In the graph the kernels read the
 * step index from device memory, so one graph serves every step. */
int dsmc_step_graph_capture(dsmc_ctx_t* ctx, const dsmc_gas_t* gas, const dsmc_path_t* path,
                            const dsmc_step_buffers_t* buf, void* stream);
/* Run the captured step for step index `step` on `stream`: same results as
 * dsmc_step(..., step, ...). */
int dsmc_step_graph_launch(dsmc_ctx_t* ctx, uint64_t step, void* stream);

/* ---------------------------------------------------------------- launch shapes
 * The block size and the number of resident blocks per SM of the kernels
 * listed below are settings of the context, chosen by dsmc_autotune_step or
 * set directly.  No setting changes a result: each of these kernels gives a
 * thread whole work items (a sorted slot, a group of cells, a pair of a
 * round, one chi) through a grid-stride loop, so every item is computed by
 * the same arithmetic in the same order whatever the shape.  (The paper
 * fixes no launch configuration; the tuned kernels are those of Sec. 2.1,
 * 2.3 and 2.5 and of the scattering integral, Sec. 3.4.) */
enum {
  DSMC_TUNE_GATHER = 0,        /* cell sort: gather of the velocities into sorted order */
  DSMC_TUNE_MOMENTS = 1,       /* cell moments */
  DSMC_TUNE_MOMENT_MATCH = 2,  /* moment matching */
  DSMC_TUNE_COLLIDE_VHS = 3,   /* VHS collide (persistent) */
  DSMC_TUNE_COLLIDE_JAGER = 4, /* Jager collide (persistent) */
  DSMC_TUNE_JAGER_CHI = 5,     /* chi batch */
  DSMC_TUNE_COLLIDE_TABLE = 6, /* look-up collide */
  DSMC_TUNE_KERNELS = 7
};

/* One launch shape and, from dsmc_autotune_step, its measured time. */
typedef struct {
  int32_t kernel;        /* DSMC_TUNE_* */
  int32_t threads;       /* threads per block: a multiple of 32 up to the kernel's limit */
  int32_t blocks_per_sm; /* blocks per SM of the grid (1..64): the grid is this many
                            blocks per SM, or fewer when the work is smaller; for the
                            persistent collides at most what the occupancy allows
                            (clamped there at launch) */
  float ms;              /* mean time of one launch, ms (0 when not measured) */
} dsmc_tune_entry_t;

/* Set (threads, blocks_per_sm) of one kernel for later launches of this
 * context; (0, 0) restores the built-in shape.  DSMC_ERR_ARG for an unknown
 * kernel, a block size that is not a multiple of 32 or above the kernel's
 * limit (the cell-moment and moment-matching kernels take 256 only), or
 * more than 64 blocks per SM.  A captured step graph keeps the
 * shapes it was captured with. */
int dsmc_tune_set(dsmc_ctx_t* ctx, int32_t kernel, int32_t threads, int32_t blocks_per_sm);
/* Current shape of one kernel (the built-in one if none was set). */
int dsmc_tune_get(dsmc_ctx_t* ctx, int32_t kernel, int32_t* threads, int32_t* blocks_per_sm);
/* Candidate shapes the autotuner tries for `kernel` (at most `cap`; *n gets
 * the count).  Host only. */
int dsmc_tune_candidates(dsmc_ctx_t* ctx, int32_t kernel, dsmc_tune_entry_t* out, int32_t cap, int32_t* n);
/* Autotune the kernels of one step of `path` on the caller's buffers: runs
 * dsmc_step once (step index `step`), then times each candidate shape of
 * the step's tunable kernels (one untimed launch, then `reps` launches
 * between CUDA events on `stream`) and keeps the fastest shape of each in
 * the context.  Synchronises `stream`.  The buffers are left holding the
 * state after an unspecified number of collide and moment-matching passes
 * over that step's pairs (each pass conserves momentum and energy), so tune
 * on a copy or before loading the state to be advanced.  trials (may be
 * NULL) receives up to `cap` measured entries; *n_trials their count. */
int dsmc_autotune_step(dsmc_ctx_t* ctx, const dsmc_gas_t* gas, const dsmc_path_t* path,
                       const dsmc_step_buffers_t* buf, uint64_t step, int32_t reps,
                       dsmc_tune_entry_t* trials, int32_t cap, int32_t* n_trials, void* stream);
/* Autotune the chi batch kernel (dsmc_jager_chi) on the caller's arrays the
 * same way; chi receives the batch's deflection angles.  Synchronises. */
int dsmc_autotune_chi(dsmc_ctx_t* ctx, const dsmc_gas_t* gas, const dsmc_potential_t* pot, int32_t n_nodes,
                      int64_t n, const float* b, const float* g, float* chi, int32_t reps,
                      dsmc_tune_entry_t* trials, int32_t cap, int32_t* n_trials, void* stream);

/* Same step from and to HOST memory: copies cell_id_host / v*_host into
 * device buffers reserved by dsmc_ctx_reserve, runs dsmc_step, copies the
 * sorted post-collision velocities and perm back, and synchronises the
 * stream.  The cell ids upload first; the velocity upload runs on a side
 * stream of the context while the cell ids are sorted, each component
 * gathered into cell order as soon as it has landed, and perm downloads
 * while the pairs are selected and updated; all of it has completed when
 * the call returns.  sigma_g_max
 * stays on the device between calls (initialised from T_cell_host on the
 * first call after a reserve).  Returns the first error, device-side ones
 * included.  Host arrays should be page-locked for the copies to overlap. */
int dsmc_ctx_reserve(dsmc_ctx_t* ctx, int32_t n_max, int32_t n_cells, int64_t capacity);
int dsmc_step_host(dsmc_ctx_t* ctx, const dsmc_gas_t* gas, const dsmc_path_t* path,
                   int32_t n, const int32_t* cell_id_host, const double* vx_host,
                   const double* vy_host, const double* vz_host, const double* T_cell_host,
                   uint64_t step, int32_t* perm_host, double* svx_host, double* svy_host,
                   double* svz_host, int64_t* n_pairs_host, void* stream);

/* ---------------------------------------------------------------- training */

/* Sec. 3.4.4 physics harvesting: target post-collision velocities of pairs
 * (vi, vj: [n x 3] FP64 row-major) deflected by chi(b, E) with azimuth eps
 * (b in Angstrom, eps in rad), as in dsmc_collide_jager. */
int dsmc_harvest_jager(dsmc_ctx_t* ctx, const dsmc_gas_t* gas, const dsmc_potential_t* pot,
                       int32_t n_nodes, int64_t n, const double* vi, const double* vj,
                       const double* b, const double* eps, double* vi_out, double* vj_out,
                       void* stream);

/* ---------------------------------------------------------------- neural operator training */

/* Parameters theta (FP32): each layer's row-major [out x in] weights,
 * concatenated, then each layer's bias (the layout of dsmc_collide_neural's
 * weights and biases).  34,563 for d_in 8, width 128, 3 hidden layers. */
int32_t dsmc_mlp_param_count(const dsmc_mlp_t* mlp);
/* Scratch of the backward kernels: one partial gradient per SM. */
size_t dsmc_train_workspace_size(dsmc_ctx_t* ctx);

/* The neural collision operator applied to a batch of n pairs (n a multiple
 * of 16) grouped in pseudo-cells of 16 consecutive pairs (32 particles):
 *   x = [v_r/sigma_v, T/T_ref, xi] (xi: Philox tag 5, counter (pair, 0, t)),
 *   y = f_theta(x) (bf16 tcgen05, weights rounded from theta),
 *   v_r' = |v_r| y/|y| (Eq. energy_shell_projection), centre-of-mass update
 *   (Sec. 2.3), moment matching of each pseudo-cell to its pre-collision
 *   momentum and energy (Sec. 2.5, centred).
 * vi, vj, vi_new, vj_new: [n x 3] FP64 row-major; T: [n] FP64.
 * Requires d_in 8, width 128, 3 hidden layers. */
int dsmc_neural_operator_forward(dsmc_ctx_t* ctx, const dsmc_mlp_t* mlp, const float* theta, uint64_t seed,
                                 uint64_t t, int64_t n, const double* vi, const double* vj, const double* T,
                                 double* vi_new, double* vj_new, void* stream);
/* Hand-written backward of the operator: given dL/dvi_new, dL/dvj_new
 * ([n x 3] FP64), writes dL/dtheta (FP32, theta layout) to grad.  The
 * moment-matching and projection backward are closed forms; the MLP
 * backward recomputes each layer's pre-activation from the saved input of
 * that layer from exactly the forward's operands (the low bf16 terms of
 * the hidden activations regenerated by running the first layers again), so
 * the recomputed pre-activations equal the forward's bit for bit, and no
 * activations are stored in HBM; dW accumulates per SM in TMEM and the
 * per-SM partials are summed in a fixed order. */
int dsmc_neural_operator_backward(dsmc_ctx_t* ctx, const dsmc_mlp_t* mlp, const float* theta, uint64_t seed,
                                  uint64_t t, int64_t n, const double* vi, const double* vj, const double* T,
                                  const double* g_vi, const double* g_vj, float* grad, void* ws,
                                  size_t ws_bytes, void* stream);
/* Loss L = mean over the 2n particles of |v_new - v_target|^2 / sigma_v^2
 * (the MSE of Sec. 2.6) and dL/dtheta in one pass; *loss (device FP64). */
int dsmc_train_loss_grad(dsmc_ctx_t* ctx, const dsmc_mlp_t* mlp, const float* theta, uint64_t seed, uint64_t t,
                         int64_t n, const double* vi, const double* vj, const double* T, const double* vi_target,
                         const double* vj_target, float* grad, double* loss, void* ws, size_t ws_bytes,
                         void* stream);
/* The stored-activation variant of dsmc_train_loss_grad, with no
 * counterpart in the paper (the check of the recomputation): the forward
 * writes every hidden layer's pre-activation accumulator (FP32, [tiles of
 * 128 pairs x 3 layers x 128 x 128]) to `act` (device memory of at least
 * dsmc_train_act_size(n) bytes, caller-owned) and the backward reads it back
 * instead of recomputing it; grad and loss equal dsmc_train_loss_grad's bit
 * for bit. */
size_t dsmc_train_act_size(int64_t n);
int dsmc_train_loss_grad_stored(dsmc_ctx_t* ctx, const dsmc_mlp_t* mlp, const float* theta, uint64_t seed,
                                uint64_t t, int64_t n, const double* vi, const double* vj, const double* T,
                                const double* vi_target, const double* vj_target, float* grad, double* loss,
                                void* ws, size_t ws_bytes, float* act, size_t act_bytes, void* stream);
/* Adam (Kingma & Ba 2015, Algorithm 1) on theta with moments m, v (FP32,
 * n_params each); step counts from 1.  The first n_weights entries are
 * weights: if weights_bf16 / biases are given, the updated weights are also
 * written as bf16 and the biases as FP32 (the collide kernel's inputs). */
int dsmc_adam_step(dsmc_ctx_t* ctx, int32_t n_params, int32_t n_weights, const float* grad, float* theta,
                   float* m, float* v, int64_t step, float lr, float beta1, float beta2, float eps,
                   uint16_t* weights_bf16, float* biases, void* stream);
/* One training step (Sec. 2.6; Adam beta = (0.9, 0.999), eps = 1e-8):
 * dsmc_train_loss_grad with noise counter t = step, then dsmc_adam_step. */
int dsmc_train_step(dsmc_ctx_t* ctx, const dsmc_mlp_t* mlp, float* theta, float* m, float* v, int64_t step,
                    float lr, uint64_t seed, int64_t n, const double* vi, const double* vj, const double* T,
                    const double* vi_target, const double* vj_target, float* grad, double* loss,
                    uint16_t* weights_bf16, float* biases, void* ws, size_t ws_bytes, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* DSMC_H_ */
