/*
 * dsmc_oracle.c -- plain, slow FP64 CPU oracle of the DSMC collision step of
 * "Physics Constrained Neural Collision Operators for VHS Surrogates and Ab
 * Initio Angle Prediction in DSMC" (arXiv 2602.21244).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  The
 * product (the CUDA library under paper_2602_21244_gb300/) never calls it and
 * shares no code, header, table or constant generator with it.
 *
 * Everything is double precision, in the order the method states, with no
 * blocking or fusion.  Compile with -ffp-contract=off so that no a*b+c is
 * fused into an FMA: the integer decisions of pair selection must be the
 * same on every host.  Built with OpenMP when the compiler has it: loops
 * over independent cells (Sec. 2.6: cells are processed in parallel),
 * independent pairs of the chi batch and independent table nodes run on
 * several threads; each cell's pairs still act one after another in
 * candidate order, so every result is the sequential one bit for bit.
 *
 * Citations are to the paper's sections and equations:
 *   Sec. 2.1   DSMC collision step, NTC rate nu ~ n sigma v_r
 *   Sec. 2.2   cell partition, NTC candidate count ~ N_k(N_k-1)(sigma v_r)_max,
 *              uniform pair draw, acceptance ~ sigma v_r; Eq. (mlp_input),
 *              Eq. (mlp_output)
 *   Sec. 2.3   Eq. (energy_shell_projection) and the centre-of-mass update
 *   Sec. 2.5   Eq. (cell_energy_clamp), cell-wise energy correction
 *   Sec. 2.6   sort by cell index, batch per cell, parallel over cells
 *   Sec. 3.4.1 Eq. (jager_potential), Eq. (damping), screened Coulomb core
 *   Sec. 3.4.2 classical scattering integral chi(b, E_r)
 *   Sec. 3.4.4 r_min = largest root, Brent-Dekker to 1e-14, u = r_min/r
 *   Sec. 3.4.4 look-up table over (b/b_max, ln E_r/k_B), bilinear interpolation
 *
 * Readings where the paper is silent (all listed in the design notes):
 *   R1  Philox4x32-10 (Salmon et al., SC'11) keyed by seed, counter
 *       (idx, cell, step_lo, tag | sub<<8 | step_hi<<16).
 *   R2  Bird's NTC constant: M~ = 1/2 N(N-1) (F_N/V_c) (sigma g)_max dt,
 *       stochastic rounding M = floor(M~ + U).
 *   R3  acceptance uses the pre-step (snapshot) velocities; (sigma g)_max is
 *       raised after the step to the largest sigma g seen among candidates.
 *   R4  accepted pairs act in candidate order on the current velocities
 *       (classical sequential DSMC).  Their "round" is 1+max(last[i],last[j]).
 *   R5  cell moment matching is centred: v <- u_pre + alpha (v - u_post),
 *       alpha = sqrt(Theta_pre/Theta_post); it equals Eq. (cell_energy_clamp)
 *       when the cell mean velocity is zero.
 *   R6  energy-shell projection divides by ||y|| (not ||y||+eps) so the pair
 *       energy is exact; ||y|| <= eps falls back to an isotropic direction.
 *   R7  the chi table of the look-up path (Sec. 3.4.4: b~ = b/b_max,
 *       E~ = ln(E_r/k_B), bilinear interpolation) has uniform nodes including
 *       both ends of each axis; E~ outside the table is clamped to it.
 *   R8  transport integrals (Eq. chapman_enskog and the two integrals after
 *       it): Q2(E) = 2 pi int_0^bmax (1 - cos^2 chi) b db with the b-integral
 *       cut at b_max; the Maxwellian average that makes Eq. (chapman_enskog)
 *       give the rigid-sphere viscosity is the Chapman-Cowling one,
 *       Omega22(T) = 1/(4 (kT)^4) int_0^inf E^3 Q2(E) exp(-E/kT) dE
 *       (the printed E^2/(2 (kT)^3) weighting would make the hard-sphere mu
 *       1.5 times the textbook value).  Both integrals by composite
 *       Gauss-Legendre rules whose nodes the caller passes: in u = (b/b_max)^2
 *       on [0, 1] and in x = E/(kT) on [0, x_max].
 *   R9  chi-MLP surrogate (Fig. nn_architecture): inputs x0 = ln(E_r)* =
 *       (ln(E_r/k_B) - ln 5)/(ln 60000 - ln 5) (min-max over the training
 *       range, as the table of R7) and x1 = b/b_max; the Softplus output is
 *       y ~ ln(1 + chi) (the training target), so chi = e^y - 1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_KB 1.380649e-23 /* Boltzmann constant, J/K (exact SI value) */
#define OR_PI 3.14159265358979323846

/* threads the parallel loops use (1 without OpenMP), and a way to set them */
int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
void or_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* Pairs of different cells share no particle.  A pair list in cell-major
 * order (pcell non-decreasing) is therefore processed cell by cell in
 * parallel, each cell's pairs one after another in their given order, which
 * is the sequential result exactly; any other order runs sequentially. */
typedef void (*or_pair_fn)(const void* ctx, int64_t p);
static void for_each_pair(int64_t n_pairs, const int32_t* pcell, or_pair_fn f, const void* ctx) {
  int cell_major = pcell != NULL;
  for (int64_t p = 1; cell_major && p < n_pairs; ++p)
    if (pcell[p] < pcell[p - 1]) cell_major = 0;
  if (!cell_major || n_pairs < 2) {
    for (int64_t p = 0; p < n_pairs; ++p) f(ctx, p);
    return;
  }
  int64_t nseg = 1;
  for (int64_t p = 1; p < n_pairs; ++p) nseg += pcell[p] != pcell[p - 1];
  int64_t* st = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nseg + 1));
  int64_t q = 0;
  st[q++] = 0;
  for (int64_t p = 1; p < n_pairs; ++p)
    if (pcell[p] != pcell[p - 1]) st[q++] = p;
  st[nseg] = n_pairs;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t g = 0; g < nseg; ++g)
    for (int64_t p = st[g]; p < st[g + 1]; ++p) f(ctx, p);
  free(st);
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, Sec. 3.3)         */
/* ------------------------------------------------------------------ */
enum { OR_TAG_NTC = 1, OR_TAG_CAND = 2, OR_TAG_ISO = 3, OR_TAG_JAGER = 4,
       OR_TAG_NOISE = 5, OR_TAG_HARVEST = 6 };

void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                      uint32_t out[4]) {
  uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k0;
    uint32_t n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
  }
  out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

static void draw(uint64_t seed, uint32_t idx, uint32_t cell, uint64_t step,
                 uint32_t tag, uint32_t sub, uint32_t out[4]) {
  uint32_t ctr[4] = {idx, cell, (uint32_t)step,
                     tag | (sub << 8) | ((uint32_t)(step >> 32) << 16)};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  or_philox4x32_10(ctr, key, out);
}

/* uniform double in [0,1) from 53 bits of two words */
double or_u53(uint32_t a, uint32_t b) {
  uint64_t x = (((uint64_t)a << 32) | b) >> 11;
  return (double)x * (1.0 / 9007199254740992.0);
}

/* integer in [0,n) by the high word of w*n (Lemire, no rejection) */
static uint32_t mulhi_n(uint32_t w, uint32_t n) {
  return (uint32_t)(((uint64_t)w * n) >> 32);
}

void or_philox_stream(uint64_t seed, uint32_t cell, uint64_t step,
                      uint32_t tag, uint32_t sub, int64_t n, uint32_t* out) {
  for (int64_t i = 0; i < n; ++i) draw(seed, (uint32_t)i, cell, step, tag, sub, out + 4 * i);
}

/* ------------------------------------------------------------------ */
/* Gas description (the oracle's own copy; the CUDA library has its   */
/* own).  Field order is the ABI order used by oracle/__init__.py.    */
/* ------------------------------------------------------------------ */
typedef struct {
  double mass;        /* kg */
  double d_ref;       /* m, VHS reference diameter */
  double omega;       /* VHS viscosity index (0.5 = hard sphere) */
  double T_ref;       /* K */
  double fn_over_vc;  /* F_N / V_c, 1/m^3 (= n / mean particles per cell) */
  double dt;          /* s */
  uint64_t seed;
  int32_t model;      /* 0: VHS cross section; 1: constant pi b_max^2 */
  int32_t pad_;
  double b_max;       /* m, impact-parameter cut-off for model 1 */
} or_gas_t;

/* Bird's VHS total cross section (Bird 1994, Eq. 4.63 form):
 *   sigma(g) = pi d_ref^2 (2 k T_ref / (m_r g^2))^(omega-1/2) / Gamma(5/2-omega),
 * m_r = m/2.  omega = 1/2 gives the hard-sphere pi d^2. */
double or_sigma(const or_gas_t* gs, double g) {
  if (gs->model == 1) return OR_PI * gs->b_max * gs->b_max;
  double mr = 0.5 * gs->mass;
  double x = 2.0 * OR_KB * gs->T_ref / (mr * g * g);
  return OR_PI * gs->d_ref * gs->d_ref * pow(x, gs->omega - 0.5) / tgamma(2.5 - gs->omega);
}

/* initial (sigma g)_max of a cell at temperature T: sigma(g0) g0 with
 * g0 = factor * sqrt(2 k T / m) */
void or_sigma_g_max_init(const or_gas_t* gs, int32_t n_cells, const double* T,
                         double factor, double* sgmax) {
  for (int32_t k = 0; k < n_cells; ++k) {
    double g0 = factor * sqrt(2.0 * OR_KB * T[k] / gs->mass);
    sgmax[k] = or_sigma(gs, g0) * g0;
  }
}

/* ------------------------------------------------------------------ */
/* Sec. 2.6 (1): stable counting sort by cell index                    */
/* ------------------------------------------------------------------ */
int or_sort_cells(int32_t n, int32_t n_cells, const int32_t* cell_id,
                  const double* vx, const double* vy, const double* vz,
                  int32_t* perm, int32_t* cell_start,
                  double* svx, double* svy, double* svz) {
  for (int32_t k = 0; k <= n_cells; ++k) cell_start[k] = 0;
  for (int32_t i = 0; i < n; ++i) {
    if (cell_id[i] < 0 || cell_id[i] >= n_cells) return -1;
    cell_start[cell_id[i] + 1] += 1;
  }
  for (int32_t k = 0; k < n_cells; ++k) cell_start[k + 1] += cell_start[k];
  int32_t* cursor = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_cells > 0 ? n_cells : 1));
  for (int32_t k = 0; k < n_cells; ++k) cursor[k] = cell_start[k];
  for (int32_t i = 0; i < n; ++i) perm[cursor[cell_id[i]]++] = i;
  free(cursor);
  for (int32_t s = 0; s < n; ++s) {
    svx[s] = vx[perm[s]]; svy[s] = vy[perm[s]]; svz[s] = vz[perm[s]];
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Cell moments, two passes: N, sum v, Theta = sum |v - u|^2, u = sum v/N */
/* ------------------------------------------------------------------ */
void or_cell_moments(int32_t n_cells, const int32_t* cs, const double* vx,
                     const double* vy, const double* vz, double* mom) {
#pragma omp parallel for schedule(dynamic, 256)
  for (int32_t k = 0; k < n_cells; ++k) {
    int32_t a = cs[k], b = cs[k + 1];
    double sx = 0, sy = 0, sz = 0;
    for (int32_t s = a; s < b; ++s) { sx += vx[s]; sy += vy[s]; sz += vz[s]; }
    double n = (double)(b - a), th = 0;
    if (b > a) {
      double ux = sx / n, uy = sy / n, uz = sz / n;
      for (int32_t s = a; s < b; ++s) {
        double dx = vx[s] - ux, dy = vy[s] - uy, dz = vz[s] - uz;
        th += dx * dx + dy * dy + dz * dz;
      }
    }
    mom[5 * k + 0] = n; mom[5 * k + 1] = sx; mom[5 * k + 2] = sy;
    mom[5 * k + 3] = sz; mom[5 * k + 4] = th;
  }
}

/* ------------------------------------------------------------------ */
/* Sec. 2.2: NTC selection, readings R2-R4                             */
/* Output pairs are cell-major in candidate order.                    */
/* ------------------------------------------------------------------ */
/* One cell k: its M candidates in order, the accepted ones with their
 * rounds.  *acc_out receives {i, j, m, round} per accepted pair (candidate
 * order, cell-local i and j), the return value their number; *best the
 * cell's raised (sigma g)_max, *rounds its number of rounds, *n_cand = M.
 * Returns -1 if M does not fit an int32. */
static int64_t select_cell(const or_gas_t* gs, int32_t k, const int32_t* cs, const double* vx,
                           const double* vy, const double* vz, const double* sgmax, uint64_t step,
                           int32_t** acc_out, double* best, int32_t* rounds, int64_t* n_cand) {
  int32_t a = cs[k], N = cs[k + 1] - cs[k];
  *acc_out = NULL; *best = sgmax[k]; *rounds = 0; *n_cand = 0;
  if (N < 2) return 0;
  uint32_t w[4];
  draw(gs->seed, 0, (uint32_t)k, step, OR_TAG_NTC, 0, w);
  double mt = 0.5 * (double)N * (double)(N - 1);
  mt = mt * gs->fn_over_vc;
  mt = mt * sgmax[k];
  mt = mt * gs->dt;
  double mf = floor(mt + or_u53(w[0], w[1]));
  if (!(mf < 2147483647.0)) return -1;
  int32_t M = (int32_t)mf;
  *n_cand = M;
  if (M == 0) return 0;
  int32_t* last = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
  int32_t* acc = (int32_t*)malloc(sizeof(int32_t) * 4 * (size_t)M);
  for (int32_t q = 0; q < N; ++q) last[q] = -1;
  int64_t na = 0;
  int32_t rmax = 0;
  for (int32_t m = 0; m < M; ++m) {
    draw(gs->seed, (uint32_t)m, (uint32_t)k, step, OR_TAG_CAND, 0, w);
    uint32_t i = mulhi_n(w[0], (uint32_t)N);
    uint32_t j = mulhi_n(w[1], (uint32_t)(N - 1));
    if (j >= i) j += 1;
    double dx = vx[a + i] - vx[a + j], dy = vy[a + i] - vy[a + j], dz = vz[a + i] - vz[a + j];
    double g = sqrt((dx * dx + dy * dy) + dz * dz);
    double sg = or_sigma(gs, g) * g;
    if (sg > *best) *best = sg;
    double U = or_u53(w[2], w[3]);
    if (U < sg / sgmax[k]) {
      int32_t r = 1 + (last[i] > last[j] ? last[i] : last[j]);
      last[i] = r; last[j] = r;
      if (r + 1 > rmax) rmax = r + 1;
      acc[4 * na + 0] = (int32_t)i; acc[4 * na + 1] = (int32_t)j;
      acc[4 * na + 2] = m; acc[4 * na + 3] = r;
      na++;
    }
  }
  free(last);
  *acc_out = acc;
  *rounds = rmax;
  return na;
}

/* The cells are independent (Sec. 2.6): each is selected on its own, then
 * the accepted pairs are concatenated in cell order and (sigma g)_max is
 * raised, so the output does not depend on the number of threads. */
int or_select_pairs(const or_gas_t* gs, int32_t n_cells, const int32_t* cs,
                    const double* vx, const double* vy, const double* vz,
                    double* sgmax, uint64_t step, int64_t capacity,
                    int32_t* pi, int32_t* pj, int32_t* pcell, int32_t* pm,
                    int32_t* pround, int64_t* n_pairs, int64_t* n_cand,
                    int32_t* n_rounds) {
  size_t nk = (size_t)(n_cells > 0 ? n_cells : 1);
  int32_t** acc = (int32_t**)calloc(nk, sizeof(int32_t*));
  int64_t* cnt = (int64_t*)calloc(nk, sizeof(int64_t));
  int64_t* cand = (int64_t*)calloc(nk, sizeof(int64_t));
  int32_t* rk = (int32_t*)calloc(nk, sizeof(int32_t));
  double* best = (double*)malloc(sizeof(double) * nk);
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(| : bad)
  for (int32_t k = 0; k < n_cells; ++k) {
    cnt[k] = select_cell(gs, k, cs, vx, vy, vz, sgmax, step, &acc[k], &best[k], &rk[k], &cand[k]);
    if (cnt[k] < 0) bad = 1;
  }
  int64_t np = 0, nc = 0;
  int32_t rmax = 0;
  for (int32_t k = 0; k < n_cells && !bad; ++k) {
    for (int64_t q = 0; q < cnt[k]; ++q) {
      if (np < capacity) {
        pi[np] = cs[k] + acc[k][4 * q]; pj[np] = cs[k] + acc[k][4 * q + 1];
        pcell[np] = k; pm[np] = acc[k][4 * q + 2]; pround[np] = acc[k][4 * q + 3];
      }
      np++;
    }
    nc += cand[k];
    if (rk[k] > rmax) rmax = rk[k];
    sgmax[k] = best[k];
  }
  for (int32_t k = 0; k < n_cells; ++k) free(acc[k]);
  free(acc); free(cnt); free(cand); free(rk); free(best);
  if (bad) return -3; /* DSMC_ERR_CAPACITY */
  *n_pairs = np; *n_cand = nc; *n_rounds = rmax;
  return np > capacity ? -3 : 0;
}

/* ------------------------------------------------------------------ */
/* Sec. 2.3: centre-of-mass pair update with a given v_r'              */
/* ------------------------------------------------------------------ */
static void pair_update(double* vx, double* vy, double* vz, int32_t i, int32_t j,
                        const double vrp[3]) {
  double cx = 0.5 * (vx[i] + vx[j]), cy = 0.5 * (vy[i] + vy[j]), cz = 0.5 * (vz[i] + vz[j]);
  vx[i] = cx + 0.5 * vrp[0]; vy[i] = cy + 0.5 * vrp[1]; vz[i] = cz + 0.5 * vrp[2];
  vx[j] = cx - 0.5 * vrp[0]; vy[j] = cy - 0.5 * vrp[1]; vz[j] = cz - 0.5 * vrp[2];
}

/* isotropic unit vector from tag 3: cos chi = 2U1-1, eps = 2 pi U2 */
static void iso_dir(uint64_t seed, int32_t cell, int32_t m, uint64_t step, double e[3]) {
  uint32_t w[4];
  draw(seed, (uint32_t)m, (uint32_t)cell, step, OR_TAG_ISO, 0, w);
  double c = 2.0 * or_u53(w[0], w[1]) - 1.0;
  double s = sqrt(1.0 - c * c);
  double ep = 2.0 * OR_PI * or_u53(w[2], w[3]);
  e[0] = c; e[1] = s * cos(ep); e[2] = s * sin(ep);
}

/* VHS isotropic scatter (the phenomenological kernel of Sec. 2.1),
 * pairs applied one after another in the given (cell-major, candidate)
 * order, reading the current velocities. */
typedef struct {
  const or_gas_t* gs;
  const int32_t *pi, *pj, *pcell, *pm;
  uint64_t step;
  double *vx, *vy, *vz;
} pairs_ctx;

static void vhs_pair(const void* c_, int64_t p) {
  const pairs_ctx* c = (const pairs_ctx*)c_;
  double *vx = c->vx, *vy = c->vy, *vz = c->vz;
  int32_t i = c->pi[p], j = c->pj[p];
  double dx = vx[i] - vx[j], dy = vy[i] - vy[j], dz = vz[i] - vz[j];
  double g = sqrt((dx * dx + dy * dy) + dz * dz);
  double e[3];
  iso_dir(c->gs->seed, c->pcell[p], c->pm[p], c->step, e);
  double vrp[3] = {g * e[0], g * e[1], g * e[2]};
  pair_update(vx, vy, vz, i, j, vrp);
}

void or_collide_vhs(const or_gas_t* gs, int64_t n_pairs, const int32_t* pi,
                    const int32_t* pj, const int32_t* pcell, const int32_t* pm,
                    uint64_t step, double* vx, double* vy, double* vz) {
  pairs_ctx c = {gs, pi, pj, pcell, pm, step, vx, vy, vz};
  for_each_pair(n_pairs, pcell, vhs_pair, &c);
}

/* ------------------------------------------------------------------ */
/* Sec. 2.5 + reading R5: centred cell moment matching                 */
/* ------------------------------------------------------------------ */
void or_moment_match(int32_t n_cells, const int32_t* cs, const double* mom_pre,
                     double* vx, double* vy, double* vz) {
#pragma omp parallel for schedule(dynamic, 256)
  for (int32_t k = 0; k < n_cells; ++k) {
    int32_t a = cs[k], b = cs[k + 1];
    if (b <= a) continue;
    double n = (double)(b - a);
    double sx = 0, sy = 0, sz = 0;
    for (int32_t s = a; s < b; ++s) { sx += vx[s]; sy += vy[s]; sz += vz[s]; }
    double ux = sx / n, uy = sy / n, uz = sz / n, th = 0;
    for (int32_t s = a; s < b; ++s) {
      double dx = vx[s] - ux, dy = vy[s] - uy, dz = vz[s] - uz;
      th += dx * dx + dy * dy + dz * dz;
    }
    double px = mom_pre[5 * k + 1] / n, py = mom_pre[5 * k + 2] / n, pz = mom_pre[5 * k + 3] / n;
    double alpha = 1.0;
    if (b - a >= 2 && th > 0.0) alpha = sqrt(mom_pre[5 * k + 4] / th);
    for (int32_t s = a; s < b; ++s) {
      vx[s] = px + alpha * (vx[s] - ux);
      vy[s] = py + alpha * (vy[s] - uy);
      vz[s] = pz + alpha * (vz[s] - uz);
    }
  }
}

/* ------------------------------------------------------------------ */
/* Sec. 3.4.1: interaction potentials, r in Angstrom, V in Kelvin      */
/* ------------------------------------------------------------------ */
typedef struct {
  int32_t kind;       /* 0 Jager form, 1 hard sphere, 2 inverse power k/r^p */
  int32_t pad_;
  double A, a1, a2, am1, am2; /* repulsive A exp(a1 r + a2 r^2 + am1/r + am2/r^2) */
  double beta;        /* Tang-Toennies damping constant ("b" in Eq. damping) */
  double C[6];        /* C6, C8, C10, C12, C14, C16 */
  double R_eps;       /* position of the well minimum; core below 0.4 R_eps */
  double At, at;      /* screened Coulomb core At exp(-at r)/r */
  double d_hs;        /* hard-sphere diameter (kind 1) */
  double kappa, p;    /* inverse power (kind 2) */
} or_pot_t;

/* Tang-Toennies damping f_n(x) = 1 - exp(-x) sum_{k=0}^{n} x^k/k!  (Eq. damping) */
double or_tt_damp(int32_t n, double x) {
  if (x > 700.0) return 1.0; /* exp(-x) x^k/k! < 1e-270 */
  double term = 1.0, sum = 1.0;
  for (int32_t k = 1; k <= n; ++k) { term *= x / (double)k; sum += term; }
  return 1.0 - exp(-x) * sum;
}

/* its derivative, f_n'(x) = exp(-x) x^n / n! */
static double tt_damp_d(int32_t n, double x) {
  if (x > 700.0) return 0.0;
  double term = 1.0;
  for (int32_t k = 1; k <= n; ++k) term *= x / (double)k;
  return exp(-x) * term;
}

double or_pot_V(const or_pot_t* P, double r) {
  if (P->kind == 1) return r < P->d_hs ? INFINITY : 0.0;
  if (P->kind == 2) return P->kappa / pow(r, P->p);
  if (r < 0.4 * P->R_eps) return P->At * exp(-P->at * r) / r;
  double rep = P->A * exp(P->a1 * r + P->a2 * r * r + P->am1 / r + P->am2 / (r * r));
  double disp = 0.0;
  for (int32_t n = 3; n <= 8; ++n)
    disp += or_tt_damp(2 * n, P->beta * r) * P->C[n - 3] / pow(r, 2.0 * n);
  return rep - disp;
}

double or_pot_dV(const or_pot_t* P, double r) {
  if (P->kind == 1) return 0.0;
  if (P->kind == 2) return -P->p * P->kappa / pow(r, P->p + 1.0);
  if (r < 0.4 * P->R_eps) return -P->At * exp(-P->at * r) * (P->at * r + 1.0) / (r * r);
  double e = P->A * exp(P->a1 * r + P->a2 * r * r + P->am1 / r + P->am2 / (r * r));
  double de = e * (P->a1 + 2.0 * P->a2 * r - P->am1 / (r * r) - 2.0 * P->am2 / (r * r * r));
  double dd = 0.0;
  for (int32_t n = 3; n <= 8; ++n) {
    double rn = pow(r, 2.0 * n);
    dd += P->C[n - 3] * (P->beta * tt_damp_d(2 * n, P->beta * r) / rn
                         - 2.0 * n * or_tt_damp(2 * n, P->beta * r) / (rn * r));
  }
  return de - dd;
}

/* Gauss-Legendre nodes on [0,1] by Newton on P_n (three-term recurrence) */
static void gauss_legendre01(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = cos(OR_PI * (i + 0.75) / (n + 0.5)), pp = 0;
    for (int it = 0; it < 100; ++it) {
      double p1 = 1.0, p2 = 0.0;
      for (int k = 1; k <= n; ++k) {
        double p3 = p2; p2 = p1;
        p1 = ((2.0 * k - 1.0) * z * p2 - (k - 1.0) * p3) / k;
      }
      pp = n * (z * p1 - p2) / (z * z - 1.0);
      double dz = p1 / pp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    x[i] = 0.5 * (1.0 - z);
    w[i] = 1.0 / ((1.0 - z * z) * pp * pp);
  }
}

/* V(r) - V(r0) for r >= r0 > 0 without cancellation: when r - r0 is small
 * relative to r0 the difference is the integral of V' over [r0, r], taken by
 * 12-point Gauss-Legendre; otherwise the plain difference. */
static double pot_dV_between(const or_pot_t* P, double r0, double dr) {
  if (P->kind == 1) return 0.0;
  double rc = 0.4 * P->R_eps;
  if (P->kind == 0 && r0 < rc && r0 + dr > rc) /* split at the core boundary */
    return pot_dV_between(P, r0, rc - r0) + pot_dV_between(P, rc, r0 + dr - rc);
  if (dr > 0.05 * r0) return or_pot_V(P, r0 + dr) - or_pot_V(P, r0);
  static _Thread_local double gx[12], gw[12];
  static _Thread_local int ready = 0;
  if (!ready) { gauss_legendre01(12, gx, gw); ready = 1; }
  double s = 0.0;
  for (int q = 0; q < 12; ++q) s += gw[q] * or_pot_dV(P, r0 + gx[q] * dr);
  return s * dr;
}

/* F(r) = 1 - b^2/r^2 - V(r)/E */
static double F_of(const or_pot_t* P, double b, double E, double r) {
  return 1.0 - (b * b) / (r * r) - or_pot_V(P, r) / E;
}

/* Brent-Dekker root finder (R. P. Brent, Algorithms for Minimization
 * Without Derivatives, 1973, ch. 4): bisection safeguarded inverse
 * quadratic / secant steps on a sign-changing bracket [a, c]. */
static double brent(const or_pot_t* P, double bb, double E, double a, double c, double rtol) {
  double fa = F_of(P, bb, E, a), fc = F_of(P, bb, E, c);
  double b = c, fb = fc;
  c = a; fc = fa;
  double d = b - a, e = d;
  for (int it = 0; it < 300; ++it) {
    if ((fb > 0 && fc > 0) || (fb < 0 && fc < 0)) { c = a; fc = fa; d = b - a; e = d; }
    if (fabs(fc) < fabs(fb)) { a = b; b = c; c = a; fa = fb; fb = fc; fc = fa; }
    double tol = 2.0 * 2.220446049250313e-16 * fabs(b) + 0.5 * rtol * fabs(b);
    double m = 0.5 * (c - b);
    if (fabs(m) <= tol || fb == 0.0) return b;
    if (fabs(e) >= tol && fabs(fa) > fabs(fb)) {
      double s = fb / fa, p, q;
      if (a == c) { p = 2.0 * m * s; q = 1.0 - s; }
      else {
        double qq = fa / fc, r = fb / fc;
        p = s * (2.0 * m * qq * (qq - r) - (b - a) * (r - 1.0));
        q = (qq - 1.0) * (r - 1.0) * (s - 1.0);
      }
      if (p > 0) q = -q; else p = -p;
      if (2.0 * p < 3.0 * m * q - fabs(tol * q) && p < fabs(0.5 * e * q)) { e = d; d = p / q; }
      else { d = m; e = m; }
    } else { d = m; e = m; }
    a = b; fa = fb;
    b += fabs(d) > tol ? d : (m > 0 ? tol : -tol);
    fb = F_of(P, bb, E, b);
  }
  return b;
}

/* Sec. 3.4.4: r_min = the largest root of F.  Scan inward on a geometric
 * grid of 4096 points from r_hi down to 0.05 A for the first F < 0, then
 * Brent to 1e-14 relative. */
double or_rmin(const or_pot_t* P, double b, double E) {
  if (P->kind == 1) return b > P->d_hs ? b : P->d_hs;
  double r_hi = 2.0 * fmax(b, P->kind == 0 ? 3.0 * P->R_eps : 1.0);
  for (int t = 0; t < 60 && F_of(P, b, E, r_hi) <= 0.0; ++t) r_hi *= 2.0;
  const double r_lo = 0.05;
  const int ngrid = 4096;
  double q = pow(r_lo / r_hi, 1.0 / (ngrid - 1));
  double r_prev = r_hi;
  for (int t = 1; t < ngrid; ++t) {
    double r = r_hi * pow(q, (double)t);
    if (F_of(P, b, E, r) < 0.0) return brent(P, b, E, r, r_prev, 1e-14);
    r_prev = r;
  }
  return NAN;
}

/* G(u) = F(r_min/u) written about r_min so that nothing cancels:
 *   G(u) = F0 + (b/r_min)^2 (1-u)(1+u) - (V(r_min/u) - V(r_min))/E,
 * given w = 1-u exactly.  F0 = F(r_min) is 0 at a root of a continuous
 * potential and 1 - (b/d)^2 at the hard-sphere wall r_min = d. */
static double G_of(const or_pot_t* P, double b, double E, double rmin, double F0, double w) {
  double u = 1.0 - w;
  double bt = b / rmin;
  double dr = rmin * w / u;
  return F0 + bt * bt * w * (1.0 + u) - pot_dV_between(P, rmin, dr) / E;
}

/* Sec. 3.4.2: chi = pi - 2 (b/r_min) int_0^1 du / sqrt(G(u)) (signed; an
 * attractive deflection is negative).  The integral has a 1/sqrt(1-u)
 * endpoint singularity; tanh-sinh quadrature (Takahasi-Mori 1974) in u
 * handles it, level doubling to 1e-14 relative. */
double or_chi(const or_pot_t* P, double b, double E) {
  if (b <= 0.0) return OR_PI;
  double rmin = or_rmin(P, b, E);
  if (!(rmin > 0.0)) return NAN;
  /* u = (1 + tanh(pi/2 sinh t))/2, 1-u = 1/(1+exp(pi sinh t)),
     du/dt = (pi/4) cosh t / cosh^2(pi/2 sinh t) */
  double F0 = P->kind == 1 ? 1.0 - (b / rmin) * (b / rmin) : 0.0;
  double h = 0.5, tmax = 4.5, prev = 0.0, est = 0.0;
  double sum = 0.0;
  int level;
  for (level = 0; level < 12; ++level) {
    double step = level == 0 ? h : 2.0 * h;
    double t0 = level == 0 ? 0.0 : h;
    for (double t = t0; t <= tmax; t += step) {
      for (int sgn = (t == 0.0 ? 1 : -1); sgn <= 1; sgn += 2) {
        double tt = sgn * t;
        double sh = OR_PI * sinh(tt);
        double w = 1.0 / (1.0 + exp(sh));          /* 1-u */
        if (w <= 0.0 || w >= 1.0) continue;
        double ch = cosh(0.5 * sh);
        double wt = 0.25 * OR_PI * cosh(tt) / (ch * ch);
        if (wt == 0.0 || !isfinite(wt)) continue;
        double G = G_of(P, b, E, rmin, F0, w);
        if (G <= 0.0) continue;
        sum += wt / sqrt(G);
      }
    }
    est = sum * h;
    if (level > 2 && fabs(est - prev) <= 1e-14 * fabs(est)) break;
    prev = est;
    h *= 0.5;
  }
  return OR_PI - 2.0 * (b / rmin) * est;
}

/* relative energy in Kelvin: E_r / k_B = (1/2) (m/2) g^2 / k_B */
static double e_kelvin(const or_gas_t* gs, double g) {
  return 0.25 * gs->mass * g * g / OR_KB;
}

/* chi(b[q], E[q]) for n independent (b, E) points, b in Angstrom, E = E_r/k_B in K */
void or_chi_many(const or_pot_t* P, int64_t n, const double* b, const double* E, double* chi) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t q = 0; q < n; ++q) chi[q] = or_chi(P, b[q], E[q]);
}

/* C1 batch: b in Angstrom, g in m/s; chi for each pair */
void or_chi_batch(const or_gas_t* gs, const or_pot_t* P, int64_t n, const double* b,
                  const double* g, double* chi) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t q = 0; q < n; ++q) chi[q] = or_chi(P, b[q], e_kelvin(gs, g[q]));
}

/* Deflect v_r by chi with azimuth eps about v_r (Bird 1994, Eq. 2.22):
 *   v_r' = cos chi v_r + g sin chi (cos eps c + sin eps a),
 *   c = (0, w, -v)/q,  a = (q^2, -u v, -u w)/(g q),  q = sqrt(v^2+w^2);
 * a = c x (v_r/g).  For q = 0 the frame is c = (0,1,0), a = c x (v_r/g). */
void or_deflect(const double vr[3], double chi, double eps, double out[3]) {
  double u = vr[0], v = vr[1], w = vr[2];
  double g = sqrt((u * u + v * v) + w * w);
  double q = sqrt(v * v + w * w);
  double cx, cy, cz, ax, ay, az;
  if (q > 1e-300 && q > 1e-12 * g) {
    cx = 0.0; cy = w / q; cz = -v / q;
    ax = q / g; ay = -u * v / (g * q); az = -u * w / (g * q);
  } else {
    cx = 0.0; cy = 1.0; cz = 0.0;
    ax = 0.0; ay = 0.0; az = u >= 0 ? -1.0 : 1.0;
  }
  double cc = cos(chi), sc = sin(chi), ce = cos(eps), se = sin(eps);
  out[0] = cc * u + g * sc * (ce * cx + se * ax);
  out[1] = cc * v + g * sc * (ce * cy + se * ay);
  out[2] = cc * w + g * sc * (ce * cz + se * az);
}

/* Jager-potential collision: b = b_max sqrt(U1) (b^2 uniform on
 * [0, b_max^2]), eps = 2 pi U2 from tag 4; chi from the scattering
 * integral; pairs in order.  chi_out (optional) receives each chi. */
typedef struct {
  pairs_ctx c;
  const or_pot_t* P;
  double* chi_out;
} jager_ctx;

static void jager_pair(const void* c_, int64_t p) {
  const jager_ctx* J = (const jager_ctx*)c_;
  const pairs_ctx* c = &J->c;
  const or_gas_t* gs = c->gs;
  double *vx = c->vx, *vy = c->vy, *vz = c->vz;
  int32_t i = c->pi[p], j = c->pj[p];
  double vr[3] = {vx[i] - vx[j], vy[i] - vy[j], vz[i] - vz[j]};
  double g = sqrt((vr[0] * vr[0] + vr[1] * vr[1]) + vr[2] * vr[2]);
  uint32_t w[4];
  draw(gs->seed, (uint32_t)c->pm[p], (uint32_t)c->pcell[p], c->step, OR_TAG_JAGER, 0, w);
  double b = gs->b_max * 1e10 * sqrt(or_u53(w[0], w[1]));
  double eps = 2.0 * OR_PI * or_u53(w[2], w[3]);
  double chi = g > 0.0 ? or_chi(J->P, b, e_kelvin(gs, g)) : 0.0;
  if (J->chi_out) J->chi_out[p] = chi;
  double vrp[3];
  if (g > 0.0) or_deflect(vr, chi, eps, vrp); else { vrp[0] = vrp[1] = vrp[2] = 0.0; }
  pair_update(vx, vy, vz, i, j, vrp);
}

void or_collide_jager(const or_gas_t* gs, const or_pot_t* P, int64_t n_pairs,
                      const int32_t* pi, const int32_t* pj, const int32_t* pcell,
                      const int32_t* pm, uint64_t step, double* vx, double* vy,
                      double* vz, double* chi_out) {
  jager_ctx J = {{gs, pi, pj, pcell, pm, step, vx, vy, vz}, P, chi_out};
  for_each_pair(n_pairs, pcell, jager_pair, &J);
}

/* The rotation and centre-of-mass update of or_collide_jager with each
 * pair's chi given (chi_in, pair order) instead of integrated, the azimuth
 * eps = 2 pi U2 from tag 4 as there: the deflection a collide kernel must
 * produce from its own chi.  vr_pre (optional, n_pairs x 3) receives each
 * pair's relative velocity before its collision, b_out (optional) its
 * impact parameter b = b_max sqrt(U1) (tag 4) in Angstrom. */
typedef struct {
  pairs_ctx c;
  const double* chi_in;
  double* vr_pre;
  double* b_out;
} given_ctx;

static void given_chi_pair(const void* c_, int64_t p) {
  const given_ctx* G = (const given_ctx*)c_;
  const pairs_ctx* c = &G->c;
  double *vx = c->vx, *vy = c->vy, *vz = c->vz;
  int32_t i = c->pi[p], j = c->pj[p];
  double vr[3] = {vx[i] - vx[j], vy[i] - vy[j], vz[i] - vz[j]};
  if (G->vr_pre) { G->vr_pre[3 * p] = vr[0]; G->vr_pre[3 * p + 1] = vr[1]; G->vr_pre[3 * p + 2] = vr[2]; }
  double g = sqrt((vr[0] * vr[0] + vr[1] * vr[1]) + vr[2] * vr[2]);
  uint32_t w[4];
  draw(c->gs->seed, (uint32_t)c->pm[p], (uint32_t)c->pcell[p], c->step, OR_TAG_JAGER, 0, w);
  double eps = 2.0 * OR_PI * or_u53(w[2], w[3]);
  if (G->b_out) G->b_out[p] = c->gs->b_max * 1e10 * sqrt(or_u53(w[0], w[1]));
  double vrp[3];
  if (g > 0.0) or_deflect(vr, G->chi_in[p], eps, vrp); else { vrp[0] = vrp[1] = vrp[2] = 0.0; }
  pair_update(vx, vy, vz, i, j, vrp);
}

void or_collide_given_chi(const or_gas_t* gs, int64_t n_pairs, const int32_t* pi, const int32_t* pj,
                          const int32_t* pcell, const int32_t* pm, uint64_t step, const double* chi_in,
                          double* vx, double* vy, double* vz, double* vr_pre, double* b_out) {
  given_ctx G = {{gs, pi, pj, pcell, pm, step, vx, vy, vz}, chi_in, vr_pre, b_out};
  for_each_pair(n_pairs, pcell, given_chi_pair, &G);
}

/* ------------------------------------------------------------------ */
/* Sec. 3.4.4 (look-up strategy): chi table and collision by look-up    */
/* ------------------------------------------------------------------ */
/* The table of the paper's look-up path, filled here by the exact chi: a
 * uniform grid in b~ = b/b_max over [0, 1] (nb nodes) and in E~ = ln(E_r/k_B)
 * over [lnE_min, lnE_max] (nE nodes), T[j nb + i] = chi(b_max i/(nb-1),
 * exp(lnE_min + j (lnE_max - lnE_min)/(nE-1))) (reading R7). */
void or_chi_table(const or_pot_t* P, double bmax_A, int32_t nb, int32_t nE, double lnE_min,
                  double lnE_max, double* T) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t j = 0; j < nE; ++j) {
    const double E = exp(lnE_min + j * (lnE_max - lnE_min) / (nE - 1));
    for (int32_t i = 0; i < nb; ++i) T[(int64_t)j * nb + i] = or_chi(P, bmax_A * i / (nb - 1), E);
  }
}

/* Bilinear interpolation in that table at (b~, E~); E~ outside the table's
 * range is clamped to it (reading R7). */
double or_chi_lookup(const float* T, int32_t nb, int32_t nE, double lnE_min, double lnE_max, double bt,
                     double lnE) {
  double x = bt * (nb - 1);
  if (x < 0.0) x = 0.0;
  if (x > nb - 1) x = nb - 1;
  double y = (lnE - lnE_min) / (lnE_max - lnE_min) * (nE - 1);
  if (y < 0.0) y = 0.0;
  if (y > nE - 1) y = nE - 1;
  int32_t i0 = (int32_t)floor(x), j0 = (int32_t)floor(y);
  if (i0 > nb - 2) i0 = nb - 2;
  if (j0 > nE - 2) j0 = nE - 2;
  const double fx = x - i0, fy = y - j0;
  const double t00 = T[(int64_t)j0 * nb + i0], t01 = T[(int64_t)j0 * nb + i0 + 1];
  const double t10 = T[(int64_t)(j0 + 1) * nb + i0], t11 = T[(int64_t)(j0 + 1) * nb + i0 + 1];
  return (1.0 - fy) * ((1.0 - fx) * t00 + fx * t01) + fy * ((1.0 - fx) * t10 + fx * t11);
}

/* Pair update with chi from the table: b~ = sqrt(U1), eps = 2 pi U2 (tag 4,
 * as the Jager path), E~ = ln(m g^2/(4 k_B)); rotation and centre-of-mass
 * update as or_collide_jager; pairs in order. */
typedef struct {
  pairs_ctx c;
  const float* T;
  int32_t nb, nE;
  double lnE_min, lnE_max;
  double* chi_out;
} table_ctx;

static void table_pair(const void* c_, int64_t p) {
  const table_ctx* L = (const table_ctx*)c_;
  const pairs_ctx* c = &L->c;
  double *vx = c->vx, *vy = c->vy, *vz = c->vz;
  int32_t i = c->pi[p], j = c->pj[p];
  double vr[3] = {vx[i] - vx[j], vy[i] - vy[j], vz[i] - vz[j]};
  double g = sqrt((vr[0] * vr[0] + vr[1] * vr[1]) + vr[2] * vr[2]);
  uint32_t w[4];
  draw(c->gs->seed, (uint32_t)c->pm[p], (uint32_t)c->pcell[p], c->step, OR_TAG_JAGER, 0, w);
  double bt = sqrt(or_u53(w[0], w[1]));
  double eps = 2.0 * OR_PI * or_u53(w[2], w[3]);
  double chi = g > 0.0 ? or_chi_lookup(L->T, L->nb, L->nE, L->lnE_min, L->lnE_max, bt, log(e_kelvin(c->gs, g)))
                       : 0.0;
  if (L->chi_out) L->chi_out[p] = chi;
  double vrp[3];
  if (g > 0.0) or_deflect(vr, chi, eps, vrp); else { vrp[0] = vrp[1] = vrp[2] = 0.0; }
  pair_update(vx, vy, vz, i, j, vrp);
}

void or_collide_table(const or_gas_t* gs, const float* T, int32_t nb, int32_t nE, double lnE_min,
                      double lnE_max, int64_t n_pairs, const int32_t* pi, const int32_t* pj,
                      const int32_t* pcell, const int32_t* pm, uint64_t step, double* vx, double* vy,
                      double* vz, double* chi_out) {
  table_ctx L = {{gs, pi, pj, pcell, pm, step, vx, vy, vz}, T, nb, nE, lnE_min, lnE_max, chi_out};
  for_each_pair(n_pairs, pcell, table_pair, &L);
}

/* ------------------------------------------------------------------ */
/* Sec. 2.2-2.3: conditional MLP + energy-shell projection             */
/* ------------------------------------------------------------------ */
typedef struct {
  int32_t d_in, width, n_hidden, d_out, act; /* act: 0 SiLU, 1 ReLU */
  int32_t pad_;
  double sigma_v, T_ref, eps;
} or_mlp_t;

/* round-to-nearest-even to bfloat16, returned as a double */
double or_bf16_round(double x) {
  float f = (float)x;
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return (double)f;
  uint32_t lsb = (u >> 16) & 1u;
  u = (u + 0x7fffu + lsb) & 0xffff0000u;
  memcpy(&f, &u, 4);
  return (double)f;
}

static double act_f(int act, double z) {
  if (act == 1) return z > 0 ? z : 0.0;
  return z / (1.0 + exp(-z));
}

/* Plain layer-by-layer forward of one sample.  W holds each layer's
 * row-major [out x in] matrix, one after another; bias likewise.  With
 * bf16 != 0 the storage precision of a bf16 tensor-core kernel is
 * emulated: the input and every hidden activation are held as the sum of
 * two bf16 terms (hi = bf16(a), lo = bf16(a - hi)). */
void or_mlp_forward1(const or_mlp_t* d, const double* W, const double* bias,
                     const double* x, int bf16, double* y) {
  double h[1024], z[1024];
  int n_in = d->d_in;
  for (int q = 0; q < n_in; ++q) {
    if (bf16) {
      double hi = or_bf16_round(x[q]);
      h[q] = hi + or_bf16_round(x[q] - hi);
    } else {
      h[q] = x[q];
    }
  }
  const double* Wl = W;
  const double* bl = bias;
  for (int l = 0; l <= d->n_hidden; ++l) {
    int n_out = l == d->n_hidden ? d->d_out : d->width;
    for (int o = 0; o < n_out; ++o) {
      double s = 0.0;
      for (int q = 0; q < n_in; ++q) s += Wl[o * n_in + q] * h[q];
      z[o] = s + bl[o];
    }
    Wl += n_out * n_in; bl += n_out;
    if (l == d->n_hidden) { for (int o = 0; o < n_out; ++o) y[o] = z[o]; break; }
    for (int o = 0; o < n_out; ++o) {
      double a = act_f(d->act, z[o]);
      if (bf16) {
        double hi = or_bf16_round(a);
        h[o] = hi + or_bf16_round(a - hi);
      } else {
        h[o] = a;
      }
    }
    n_in = n_out;
  }
}

void or_mlp_forward(const or_mlp_t* d, const double* W, const double* bias, int64_t n,
                    const double* x, int bf16, double* y) {
#pragma omp parallel for schedule(static)
  for (int64_t s = 0; s < n; ++s) or_mlp_forward1(d, W, bias, x + s * d->d_in, bf16, y + s * d->d_out);
}

/* Box-Muller pair from two uniforms: rho = sqrt(-2 ln(1-U1)), theta = 2 pi U2 */
static void box_muller(double u1, double u2, double* z0, double* z1) {
  double rho = sqrt(-2.0 * log(1.0 - u1));
  double th = 2.0 * OR_PI * u2;
  *z0 = rho * cos(th); *z1 = rho * sin(th);
}

/* latent noise xi (Sec. 2.2): four N(0,1) values from tag 5, subs 0 and 1 */
void or_noise4(uint64_t seed, int32_t cell, int32_t m, uint64_t step, double z[4]) {
  uint32_t wa[4], wb[4];
  draw(seed, (uint32_t)m, (uint32_t)cell, step, OR_TAG_NOISE, 0, wa);
  draw(seed, (uint32_t)m, (uint32_t)cell, step, OR_TAG_NOISE, 1, wb);
  box_muller(or_u53(wa[0], wa[1]), or_u53(wa[2], wa[3]), &z[0], &z[1]);
  box_muller(or_u53(wb[0], wb[1]), or_u53(wb[2], wb[3]), &z[2], &z[3]);
}

/* MLP input of Eq. (mlp_input): [v_r/sigma_v, (T_cell/T_ref), xi] */
void or_neural_features(const or_mlp_t* d, const double vr[3], double T_cell,
                        const double z[4], double* x) {
  x[0] = vr[0] / d->sigma_v; x[1] = vr[1] / d->sigma_v; x[2] = vr[2] / d->sigma_v;
  if (d->d_in == 8) { x[3] = T_cell / d->T_ref; x[4] = z[0]; x[5] = z[1]; x[6] = z[2]; x[7] = z[3]; }
  else { x[3] = z[0]; x[4] = z[1]; x[5] = z[2]; }
}

/* Neural collision: features, MLP, projection (reading R6), CM update,
 * pairs in order.  T_cell of a cell = m Theta_pre / (3 k_B N).  u_out
 * (optional) receives each pair's unit direction. */
typedef struct {
  pairs_ctx c;
  const or_mlp_t* d;
  const double *W, *bias, *mom_pre;
  int bf16;
  double* u_out;
} neural_ctx;

static void neural_pair(const void* c_, int64_t p) {
  const neural_ctx* Nc = (const neural_ctx*)c_;
  const pairs_ctx* c = &Nc->c;
  const or_gas_t* gs = c->gs;
  const or_mlp_t* d = Nc->d;
  double *vx = c->vx, *vy = c->vy, *vz = c->vz;
  int32_t i = c->pi[p], j = c->pj[p], k = c->pcell[p];
  double vr[3] = {vx[i] - vx[j], vy[i] - vy[j], vz[i] - vz[j]};
  double g = sqrt((vr[0] * vr[0] + vr[1] * vr[1]) + vr[2] * vr[2]);
  double T = gs->mass * Nc->mom_pre[5 * k + 4] / (3.0 * OR_KB * Nc->mom_pre[5 * k + 0]);
  double z[4], x[8], y[3];
  or_noise4(gs->seed, k, c->pm[p], c->step, z);
  or_neural_features(d, vr, T, z, x);
  or_mlp_forward1(d, Nc->W, Nc->bias, x, Nc->bf16, y);
  double ny = sqrt((y[0] * y[0] + y[1] * y[1]) + y[2] * y[2]);
  double e[3];
  if (ny > d->eps) { e[0] = y[0] / ny; e[1] = y[1] / ny; e[2] = y[2] / ny; }
  else iso_dir(gs->seed, k, c->pm[p], c->step, e);
  if (Nc->u_out) { Nc->u_out[3 * p] = e[0]; Nc->u_out[3 * p + 1] = e[1]; Nc->u_out[3 * p + 2] = e[2]; }
  double vrp[3] = {g * e[0], g * e[1], g * e[2]};
  pair_update(vx, vy, vz, i, j, vrp);
}

void or_collide_neural(const or_gas_t* gs, const or_mlp_t* d, const double* W,
                       const double* bias, const double* mom_pre, int64_t n_pairs,
                       const int32_t* pi, const int32_t* pj, const int32_t* pcell,
                       const int32_t* pm, uint64_t step, int bf16, double* vx,
                       double* vy, double* vz, double* u_out) {
  neural_ctx Nc = {{gs, pi, pj, pcell, pm, step, vx, vy, vz}, d, W, bias, mom_pre, bf16, u_out};
  for_each_pair(n_pairs, pcell, neural_pair, &Nc);
}

/* Jager harvest of training targets (Sec. 3.4.4 "physics harvesting"):
 * per pair, deflect v_r = v_i - v_j by chi(b, E) with azimuth eps and
 * apply the CM update.  b in Angstrom. */
void or_harvest_jager(const or_gas_t* gs, const or_pot_t* P, int64_t n,
                      const double* vi, const double* vj, const double* b,
                      const double* eps, double* vi_out, double* vj_out) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t p = 0; p < n; ++p) {
    double vr[3] = {vi[3 * p] - vj[3 * p], vi[3 * p + 1] - vj[3 * p + 1], vi[3 * p + 2] - vj[3 * p + 2]};
    double g = sqrt((vr[0] * vr[0] + vr[1] * vr[1]) + vr[2] * vr[2]);
    double chi = or_chi(P, b[p], e_kelvin(gs, g));
    double vrp[3];
    or_deflect(vr, chi, eps[p], vrp);
    for (int c = 0; c < 3; ++c) {
      double cm = 0.5 * (vi[3 * p + c] + vj[3 * p + c]);
      vi_out[3 * p + c] = cm + 0.5 * vrp[c];
      vj_out[3 * p + c] = cm - 0.5 * vrp[c];
    }
  }
}

/* ------------------------------------------------------------------ */
/* Macroscopic validation: transport cross-section, Omega(2,2), mu(T)   */
/* (Eq. chapman_enskog and the two integrals after it; reading R8)      */
/* ------------------------------------------------------------------ */

/* Q2(E) in m^2 for E = E_r/k_B in Kelvin, b_max in Angstrom:
 * Q2 = 2 pi int_0^bmax sin^2 chi b db = pi bmax^2 int_0^1 sin^2 chi(bmax sqrt(u), E) du,
 * by the rule (u[k], wu[k]), k < nb, on [0, 1]. */
double or_transport_q2(const or_pot_t* P, double E, double bmax, int32_t nb, const double* u,
                       const double* wu) {
  double acc = 0.0;
  for (int32_t k = 0; k < nb; ++k) {
    double chi = or_chi(P, bmax * sqrt(u[k]), E);
    double s = sin(chi);
    acc += wu[k] * (s * s);
  }
  return OR_PI * bmax * bmax * acc * 1e-20;
}

/* Omega22(T) (m^2) and mu(T) (Pa s) for n_T temperatures; the x-rule
 * (x[j], wx[j]), j < nx, integrates over x = E/(kT) on [0, x_max]:
 * Omega22 = 1/4 int x^3 exp(-x) Q2(x T) dx,  mu = 5/16 sqrt(pi m k T) / Omega22. */
void or_transport_viscosity(const or_pot_t* P, double mass, int32_t n_T, const double* T, double bmax,
                            int32_t nb, const double* u, const double* wu, int32_t nx, const double* x,
                            const double* wx, double* omega22, double* mu) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t i = 0; i < n_T; ++i) {
    double om = 0.0;
    for (int32_t j = 0; j < nx; ++j) {
      double q = or_transport_q2(P, x[j] * T[i], bmax, nb, u, wu);
      om += wx[j] * x[j] * x[j] * x[j] * exp(-x[j]) * q;
    }
    om *= 0.25;
    omega22[i] = om;
    mu[i] = 5.0 / 16.0 * sqrt(OR_PI * mass * OR_KB * T[i]) / om;
  }
}

/* ------------------------------------------------------------------ */
/* chi-MLP surrogate (Fig. nn_architecture; reading R9)                 */
/* ------------------------------------------------------------------ */
static const int32_t or_chi_dims[7] = {2, 512, 512, 512, 256, 128, 1};

static double or_softplus(double z) { return fmax(z, 0.0) + log1p(exp(-fabs(z))); }

/* y = Softplus(W6 h5 + b6), h_l = SiLU(W_l h_{l-1} + b_l), h0 = x; W row-major
 * [out x in] per layer, concatenated; bias concatenated.  emul != 0 emulates
 * the storage of a bf16 tensor-core kernel: the input as two bf16 terms
 * (hi + lo), the activations of hidden layers 1-4 rounded to bf16 once, the
 * fifth hidden layer's activations exact (an FP32 dot product follows). */
void or_chi_mlp_forward(const double* W, const double* bias, int64_t n, const double* x, int emul, double* y) {
#pragma omp parallel
  {
  double* a = (double*)malloc(sizeof(double) * 512);
  double* b = (double*)malloc(sizeof(double) * 512);
#pragma omp for schedule(dynamic, 16)
  for (int64_t s = 0; s < n; ++s) {
    for (int q = 0; q < 2; ++q) {
      double v = x[2 * s + q];
      if (emul) { double hi = or_bf16_round(v); v = hi + or_bf16_round(v - hi); }
      a[q] = v;
    }
    const double* w = W;
    const double* bb = bias;
    for (int l = 0; l < 6; ++l) {
      const int din = or_chi_dims[l], dout = or_chi_dims[l + 1];
      for (int o = 0; o < dout; ++o) {
        double z = bb[o];
        for (int i = 0; i < din; ++i) z += w[(int64_t)o * din + i] * a[i];
        if (l < 5) {
          double h = z / (1.0 + exp(-z));
          if (emul && l < 4) h = or_bf16_round(h);
          b[o] = h;
        } else {
          y[s] = or_softplus(z);
        }
      }
      w += (int64_t)din * dout;
      bb += dout;
      double* t = a; a = b; b = t;
    }
  }
  free(a);
  free(b);
  }
}
