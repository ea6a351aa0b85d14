/*
 * oracle.c -- plain FP64 CPU oracle (test infrastructure only; see oracle.h).
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared oracle.c -lm -lpthread
 * (oracle/__init__.py does this).  Threads only split loops whose iterations
 * are independent (paths in the forward pass, strikes in the backward pass),
 * so every result is identical for any thread count.
 */
#include "oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10.  The paper's inputs are two doubles per path, asset and    */
/* step produced on the host (Sec. 2.2.1); here they come from a counter-    */
/* based generator.  Round function and constants: Salmon, Moraes, Dror,     */
/* Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11.              */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t prod0 = (uint64_t)M0 * (uint64_t)x0;
    uint64_t prod1 = (uint64_t)M1 * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += W0;  /* key schedule: the key advances by the Weyl constants */
    k1 += W1;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ------------------------------------------------------------------------ */
/* Uniforms on exact symmetric grids (never 0 or 1, so the quantile is      */
/* finite and quantile(1 - u) = -quantile(u) holds exactly).                */
/* ------------------------------------------------------------------------ */
double orc_uniform_f64(uint32_t hi, uint32_t lo) {
  uint64_t m = ((uint64_t)hi << 20) | (uint64_t)(lo >> 12); /* 52 bits */
  return ((double)m + 0.5) * 0x1p-52;
}

double orc_uniform_f32(uint32_t w) {
  uint32_t m = w >> 9; /* 23 bits */
  return ((double)m + 0.5) * 0x1p-23;
}

/* ------------------------------------------------------------------------ */
/* Rounding to a narrower binary floating-point format, to nearest with     */
/* ties to even, from the format's definition: p significant bits, normal   */
/* exponents emin..emax (a value below 2^emin is a multiple of the smallest */
/* subnormal 2^(emin - p + 1)), anything that rounds above the largest      */
/* finite value (2 - 2^(1 - p)) 2^emax becomes infinite.  IEEE binary16:    */
/* p = 11, emin = -14, emax = 15; bfloat16: p = 8, emin = -126, emax = 127. */
/* Used for the reduced-precision path store (the paper's study of data     */
/* types, Sec. 4.2 and Table 4, applied to storage).                      */
/* ------------------------------------------------------------------------ */
static double orc_round_format(double x, int p, int emin, int emax) {
  if (x != x || x == 0.0 || isinf(x)) return x;
  const double a = fabs(x);
  int e;
  frexp(a, &e);          /* a = f 2^e with f in [1/2, 1): leading bit 2^(e-1) */
  int E = e - 1;
  if (E < emin) E = emin; /* subnormal range: the quantum stays 2^(emin-p+1) */
  const double q = ldexp(1.0, E - p + 1);  /* spacing of the format near a */
  const double r = a / q;                   /* exact: q is a power of two */
  const double fl = floor(r), frac = r - fl;
  double n;
  if (frac > 0.5) n = fl + 1.0;
  else if (frac < 0.5) n = fl;
  else n = fmod(fl, 2.0) == 0.0 ? fl : fl + 1.0;  /* tie: the even neighbour */
  double res = n * q;
  if (res > ldexp(2.0 - ldexp(1.0, 1 - p), emax)) res = INFINITY;
  return copysign(res, x);
}

double orc_round_f16(double x) { return orc_round_format(x, 11, -14, 15); }
double orc_round_bf16(double x) { return orc_round_format(x, 8, -126, 127); }
void orc_round_n(const double* x, double* y, size_t n, int store) {
  for (size_t i = 0; i < n; ++i) y[i] = store == 1 ? orc_round_f16(x[i]) : orc_round_bf16(x[i]);
}

/* ------------------------------------------------------------------------ */
/* Normal quantile from its definition: Phi(z) = erfc(-z / sqrt 2) / 2,     */
/* and z(u) is the root of Phi(z) = u.  Newton's method inside a bracket   */
/* that always holds the root (bisection when a step leaves it).            */
/* ------------------------------------------------------------------------ */
static double orc_phi_cdf(double z) { return 0.5 * erfc(-z / sqrt(2.0)); }

/* Phi(z) - u.  Near the centre (u > 1/4) the same quantity is formed as
 * erf(z / sqrt 2) / 2 - (u - 1/2), whose terms carry relative accuracy
 * (u - 1/2 is exact there), so the root keeps full relative precision. */
static double orc_phi_minus(double z, double u) {
  if (u > 0.25) return 0.5 * erf(z / sqrt(2.0)) - (u - 0.5);
  return orc_phi_cdf(z) - u;
}

static double orc_phi_pdf(double z) {
  return exp(-0.5 * z * z) / sqrt(2.0 * 3.14159265358979323846);
}

double orc_norm_inv(double u) {
  if (!(u > 0.0 && u < 1.0)) return NAN;
  if (u > 0.5) return -orc_norm_inv(1.0 - u); /* 1 - u is exact here */
  if (u == 0.5) return 0.0;
  double lo = -40.0, hi = 0.0; /* Phi(lo) < u < Phi(hi) */
  double z = -sqrt(-2.0 * log(u));
  if (!(z > lo)) z = 0.5 * (lo + hi);
  for (int it = 0; it < 200; ++it) {
    double f = orc_phi_minus(z, u);
    if (f == 0.0) return z;
    if (f > 0.0) hi = z; else lo = z;
    double step = f / orc_phi_pdf(z);
    double zn = z - step;
    if (!(zn > lo && zn < hi)) zn = 0.5 * (lo + hi);
    double dz = fabs(zn - z);
    z = zn;
    if (dz <= 0x1p-54 * fabs(z) || hi - lo <= 0x1p-54 * fabs(z)) break;
  }
  return z;
}

/* The random inputs of one step (Sec. 2.2.1: two random numbers per path,
 * asset and time step).  Counter (path, step, stream, 0), key = seed.
 * U_V feeds both branches of the QE variance step; Z_X drives the log price. */
void orc_draws(uint64_t seed, uint32_t stream, uint32_t path, uint32_t step,
               int grid, double out[3]) {
  orc_draws_asset(seed, stream, path, step, 0u, grid, out);
}

void orc_draws_asset(uint64_t seed, uint32_t stream, uint32_t path, uint32_t step,
                     uint32_t asset, int grid, double out[3]) {
  uint32_t ctr[4] = {path, step, stream, asset};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t w[4];
  orc_philox4x32_10(ctr, key, w);
  double uV, uX;
  if (grid == ORC_GRID_F32) {
    uV = orc_uniform_f32(w[0]);
    uX = orc_uniform_f32(w[2]);
  } else {
    uV = orc_uniform_f64(w[0], w[1]);
    uX = orc_uniform_f64(w[2], w[3]);
  }
  out[0] = uV;
  out[1] = orc_norm_inv(uV);
  out[2] = orc_norm_inv(uX);
}

/* ------------------------------------------------------------------------ */
/* Heston discretisations.  The paper's path generation follows Andersen's  */
/* QE method for the Heston model (Sec. 2.2; variance then log price, then */
/* the exponential, Sec. 2.2.1 and Sec. 4.1 Listings 1-2).                  */
/* ------------------------------------------------------------------------ */
void orc_qe_step(const orc_heston* m, double dt, double x, double v,
                 double uV, double zV, double zX, double out[2]) {
  const double kappa = m->kappa, theta = m->theta, xi = m->xi, rho = m->rho;
  const double E = exp(-kappa * dt);
  /* conditional mean and variance of v(t + dt) given v(t) */
  const double mean = theta + (v - theta) * E;
  const double var = v * xi * xi * E * (1.0 - E) / kappa +
                     theta * xi * xi * (1.0 - E) * (1.0 - E) / (2.0 * kappa);
  const double psi = var / (mean * mean);
  double v1;
  if (psi <= 1.5) {
    /* quadratic branch: v1 = a (b + Z_V)^2 */
    const double inv = 2.0 / psi;
    const double b2 = inv - 1.0 + sqrt(inv) * sqrt(inv - 1.0);
    const double b = sqrt(b2);
    const double a = mean / (1.0 + b2);
    v1 = a * (b + zV) * (b + zV);
  } else {
    /* exponential branch: mass p at zero, exponential tail of rate beta */
    const double p = (psi - 1.0) / (psi + 1.0);
    const double beta = (1.0 - p) / mean;
    v1 = (uV <= p) ? 0.0 : log((1.0 - p) / (1.0 - uV)) / beta;
  }
  /* log-price step with gamma1 = gamma2 = 1/2 and no martingale correction */
  const double K0 = -rho * kappa * theta * dt / xi;
  const double K1 = 0.5 * dt * (kappa * rho / xi - 0.5) - rho / xi;
  const double K2 = 0.5 * dt * (kappa * rho / xi - 0.5) + rho / xi;
  const double K3 = 0.5 * dt * (1.0 - rho * rho);
  const double K4 = 0.5 * dt * (1.0 - rho * rho);
  const double x1 = x + (m->r - m->q) * dt + K0 + K1 * v + K2 * v1 +
                    sqrt(K3 * v + K4 * v1) * zX;
  out[0] = x1;
  out[1] = v1;
}

void orc_ft_step(const orc_heston* m, double dt, double x, double v,
                 double zV, double zX, double out[3]) {
  const double vp = v > 0.0 ? v : 0.0; /* full truncation */
  const double v1 = v + m->kappa * (m->theta - vp) * dt +
                    m->xi * sqrt(vp * dt) * zV;
  const double x1 = x + (m->r - m->q - 0.5 * vp) * dt +
                    sqrt(vp * dt) * (m->rho * zV +
                                     sqrt(1.0 - m->rho * m->rho) * zX);
  out[0] = x1;
  out[1] = v1;
  out[2] = v1 > 0.0 ? v1 : 0.0;
}

static int orc_model_ok(const orc_heston* m, double T, int scheme) {
  const double vals[9] = {m->S0, m->r, m->q, m->v0, m->kappa, m->theta,
                          m->xi, m->rho, T};
  for (int i = 0; i < 9; ++i)
    if (!isfinite(vals[i])) return 0;
  if (!(m->S0 > 0.0) || !(T > 0.0) || m->v0 < 0.0 || !(m->kappa > 0.0) ||
      !(m->theta > 0.0) || m->xi < 0.0 || fabs(m->rho) > 1.0)
    return 0;
  if (scheme == ORC_QE && !(m->xi > 0.0)) return 0;
  if (scheme != ORC_QE && scheme != ORC_FT_EULER) return 0;
  return 1;
}

/* ---- a tiny parallel-for over independent iterations ------------------- */
typedef void (*orc_body)(void* ctx, uint32_t i);
typedef struct {
  orc_body fn;
  void* ctx;
  uint32_t n, tid, nt;
} orc_job;

static void* orc_worker(void* arg) {
  orc_job* j = (orc_job*)arg;
  for (uint32_t i = j->tid; i < j->n; i += j->nt) j->fn(j->ctx, i);
  return NULL;
}

static void orc_parallel_for(uint32_t n, int n_threads, orc_body fn,
                             void* ctx) {
  if (n_threads < 1) n_threads = 1;
  if ((uint32_t)n_threads > n) n_threads = (int)(n ? n : 1);
  if (n_threads == 1) {
    for (uint32_t i = 0; i < n; ++i) fn(ctx, i);
    return;
  }
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * n_threads);
  orc_job* jobs = (orc_job*)malloc(sizeof(orc_job) * n_threads);
  int started = 0;
  for (int t = 0; t < n_threads; ++t) {
    jobs[t].fn = fn; jobs[t].ctx = ctx; jobs[t].n = n;
    jobs[t].tid = (uint32_t)t; jobs[t].nt = (uint32_t)n_threads;
    if (pthread_create(&th[t], NULL, orc_worker, &jobs[t]) != 0) break;
    ++started;
  }
  if (started < n_threads) {
    /* run the missing threads' shares inline */
    for (int t = started; t < n_threads; ++t) orc_worker(&jobs[t]);
  }
  for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
  free(th);
  free(jobs);
}

/* ---- forward pass: paths x time steps ---------------------------------- */
typedef struct {
  const orc_heston* m;
  double dt;
  int scheme, grid;
  uint32_t P, N, stream;
  uint64_t seed;
  double *S, *V;
} orc_paths_ctx;

#define ORC_CHUNK 1024u

static void orc_paths_chunk(void* vctx, uint32_t chunk) {
  const orc_paths_ctx* c = (const orc_paths_ctx*)vctx;
  uint32_t p0 = chunk * ORC_CHUNK;
  uint32_t p1 = p0 + ORC_CHUNK < c->P ? p0 + ORC_CHUNK : c->P;
  for (uint32_t p = p0; p < p1; ++p) {
    double x = 0.0; /* log(S / S0) */
    double v = c->m->v0;
    c->S[p] = c->m->S0;
    c->V[p] = c->m->v0;
    for (uint32_t n = 0; n < c->N; ++n) {
      double d[3];
      orc_draws(c->seed, c->stream, p, n, c->grid, d);
      double stored_v;
      if (c->scheme == ORC_QE) {
        double o[2];
        orc_qe_step(c->m, c->dt, x, v, d[0], d[1], d[2], o);
        x = o[0]; v = o[1]; stored_v = v;
      } else {
        double o[3];
        orc_ft_step(c->m, c->dt, x, v, d[1], d[2], o);
        x = o[0]; v = o[1]; stored_v = o[2];
      }
      /* exponential of the log price (Sec. 2.2.1) */
      c->S[(size_t)(n + 1) * c->P + p] = c->m->S0 * exp(x);
      c->V[(size_t)(n + 1) * c->P + p] = stored_v;
    }
  }
}

int orc_path_one(const orc_heston* m, double T, int scheme, int grid,
                 uint32_t path, uint32_t N, uint64_t seed, uint32_t stream,
                 double* S, double* V) {
  if (!m || !S || !V || N == 0) return -1;
  if (!orc_model_ok(m, T, scheme)) return -1;
  if (grid != ORC_GRID_F64 && grid != ORC_GRID_F32) return -1;
  /* the chunked forward pass restricted to one path: same arithmetic */
  orc_paths_ctx c = {m, T / (double)N, scheme, grid, 1u, N, stream, seed, S, V};
  double x = 0.0, v = m->v0;
  S[0] = m->S0;
  V[0] = m->v0;
  for (uint32_t n = 0; n < N; ++n) {
    double d[3];
    orc_draws(seed, stream, path, n, grid, d);
    if (scheme == ORC_QE) {
      double o[2];
      orc_qe_step(m, c.dt, x, v, d[0], d[1], d[2], o);
      x = o[0]; v = o[1];
      V[n + 1] = v;
    } else {
      double o[3];
      orc_ft_step(m, c.dt, x, v, d[1], d[2], o);
      x = o[0]; v = o[1];
      V[n + 1] = o[2];
    }
    S[n + 1] = m->S0 * exp(x);
  }
  return 0;
}

int orc_paths(const orc_heston* m, double T, int scheme, int grid,
              uint32_t P, uint32_t N, uint64_t seed, uint32_t stream,
              double* S, double* V, int n_threads) {
  if (!m || !S || !V || P == 0 || N == 0) return -1;
  if (!orc_model_ok(m, T, scheme)) return -1;
  if (grid != ORC_GRID_F64 && grid != ORC_GRID_F32) return -1;
  orc_paths_ctx c = {m, T / (double)N, scheme, grid, P, N, stream, seed, S, V};
  uint32_t chunks = (P + ORC_CHUNK - 1) / ORC_CHUNK;
  orc_parallel_for(chunks, n_threads, orc_paths_chunk, &c);
  return 0;
}

/* ---- STAC-A2 multi-asset path reduction (Sec. 2.2.1, Sec. 4.1) --------- */
/* Each asset of a path follows its own Heston model with its own random     */
/* inputs (two per path, asset and date); the Longstaff-Schwartz path        */
/* reduction keeps, for every path and date, the largest asset value.        */

/* common factor of the log-price shocks of path `path` at date `step` */
static double orc_common_shock(uint64_t seed, uint32_t stream, uint32_t path,
                               uint32_t step, int grid) {
  uint32_t ctr[4] = {path, step, stream, 0xFFFFFFFFu};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t w[4];
  orc_philox4x32_10(ctr, key, w);
  const double u = grid == ORC_GRID_F32 ? orc_uniform_f32(w[2]) : orc_uniform_f64(w[2], w[3]);
  return orc_norm_inv(u);
}

/* one date of one asset: x, v advanced in place, returns S */
static double orc_asset_step(const orc_heston* m, double dt, int scheme, int grid,
                             double rho_assets, uint64_t seed, uint32_t stream,
                             uint32_t path, uint32_t n, uint32_t asset, double* x,
                             double* v) {
  double d[3];
  orc_draws_asset(seed, stream, path, n, asset, grid, d);
  double zX = d[2];
  if (rho_assets > 0.0) {
    const double zc = orc_common_shock(seed, stream, path, n, grid);
    zX = sqrt(rho_assets) * zc + sqrt(1.0 - rho_assets) * d[2];
  }
  if (scheme == ORC_QE) {
    double o[2];
    orc_qe_step(m, dt, *x, *v, d[0], d[1], zX, o);
    *x = o[0]; *v = o[1];
  } else {
    double o[3];
    orc_ft_step(m, dt, *x, *v, d[1], zX, o);
    *x = o[0]; *v = o[1];
  }
  return m->S0 * exp(*x);
}

typedef struct {
  const orc_heston* models;
  uint32_t A, P, N, stream;
  double dt, rho;
  int scheme, grid;
  uint64_t seed;
  double* M;
} orc_multi_ctx;

static void orc_multi_chunk(void* vctx, uint32_t chunk) {
  const orc_multi_ctx* c = (const orc_multi_ctx*)vctx;
  uint32_t p0 = chunk * ORC_CHUNK;
  uint32_t p1 = p0 + ORC_CHUNK < c->P ? p0 + ORC_CHUNK : c->P;
  double* x = (double*)malloc(sizeof(double) * c->A);
  double* v = (double*)malloc(sizeof(double) * c->A);
  for (uint32_t p = p0; p < p1; ++p) {
    double m0 = c->models[0].S0;
    for (uint32_t a = 0; a < c->A; ++a) {
      x[a] = 0.0;
      v[a] = c->models[a].v0;
      if (c->models[a].S0 > m0) m0 = c->models[a].S0;
    }
    c->M[p] = m0;
    for (uint32_t n = 0; n < c->N; ++n) {
      double mx = 0.0;
      for (uint32_t a = 0; a < c->A; ++a) {
        const double S = orc_asset_step(&c->models[a], c->dt, c->scheme, c->grid, c->rho,
                                        c->seed, c->stream, p, n, a, &x[a], &v[a]);
        if (a == 0 || S > mx) mx = S;
      }
      c->M[(size_t)(n + 1) * c->P + p] = mx;
    }
  }
  free(x);
  free(v);
}

int orc_multi_max(const orc_heston* models, uint32_t A, double T, int scheme, int grid,
                  double rho_assets, uint32_t P, uint32_t N, uint64_t seed,
                  uint32_t stream, double* M, int n_threads) {
  if (!models || !M || A == 0 || P == 0 || N == 0) return -1;
  if (!(rho_assets >= 0.0 && rho_assets <= 1.0)) return -1;
  if (grid != ORC_GRID_F64 && grid != ORC_GRID_F32) return -1;
  for (uint32_t a = 0; a < A; ++a)
    if (!orc_model_ok(&models[a], T, scheme)) return -1;
  orc_multi_ctx c = {models, A, P, N, stream, T / (double)N, rho_assets, scheme, grid, seed, M};
  uint32_t chunks = (P + ORC_CHUNK - 1) / ORC_CHUNK;
  orc_parallel_for(chunks, n_threads, orc_multi_chunk, &c);
  return 0;
}

int orc_asset_path(const orc_heston* m, uint32_t asset, double T, int scheme, int grid,
                   double rho_assets, uint32_t path, uint32_t N, uint64_t seed,
                   uint32_t stream, double* S) {
  if (!m || !S || N == 0) return -1;
  if (!(rho_assets >= 0.0 && rho_assets <= 1.0)) return -1;
  if (!orc_model_ok(m, T, scheme)) return -1;
  double x = 0.0, v = m->v0;
  S[0] = m->S0;
  for (uint32_t n = 0; n < N; ++n)
    S[n + 1] = orc_asset_step(m, T / (double)N, scheme, grid, rho_assets, seed, stream, path,
                              n, asset, &x, &v);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Longstaff-Schwartz backward induction (Sec. 2.2: Longstaff and Schwartz  */
/* for early exercise; Sec. 2.2.1: a reduction followed by a quadratic      */
/* curve fit).  Readings: exercise dates t_1..t_N; in-the-money means a     */
/* strictly positive payoff; only those paths enter the regression; the     */
/* basis is scaled and centred, x = S/K - 1 and w = v/theta - 1 (the same   */
/* fitted function as the raw monomials of S and v, with normal equations  */
/* far better conditioned); the regression target is the                    */
/* cash flow discounted to the current date; exercise when the payoff       */
/* strictly exceeds the fitted continuation value; a date with fewer        */
/* in-the-money paths than basis functions, or a Cholesky pivot at or       */
/* below 1e-13 times the largest diagonal entry, has no exercise.           */
/* ------------------------------------------------------------------------ */
static double orc_payoff(int type, double K, double s) {
  double h = (type == ORC_PUT) ? K - s : s - K;
  return h > 0.0 ? h : 0.0;
}

static int orc_basis(int basis, double s, double v, double K, double theta,
                     double phi[6]) {
  const double x = s / K - 1.0, w = v / theta - 1.0;
  phi[0] = 1.0;
  phi[1] = x;
  phi[2] = x * x;
  if (basis == ORC_BASIS_S2) return 3;
  phi[3] = w;
  phi[4] = x * w;
  phi[5] = w * w;
  return 6;
}

/* Solve A beta = c (A symmetric positive definite, B x B) by Cholesky.
 * Returns 0, or -1 when a pivot falls to the singular threshold. */
static int orc_cholesky_solve(int B, const double A[6][6], const double c[6],
                              double beta[6]) {
  double L[6][6] = {{0}};
  double maxdiag = 0.0;
  for (int i = 0; i < B; ++i)
    if (A[i][i] > maxdiag) maxdiag = A[i][i];
  for (int j = 0; j < B; ++j) {
    double d = A[j][j];
    for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
    if (!(d > 1e-13 * maxdiag)) return -1;
    L[j][j] = sqrt(d);
    for (int i = j + 1; i < B; ++i) {
      double s = A[i][j];
      for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
      L[i][j] = s / L[j][j];
    }
  }
  double z[6];
  for (int i = 0; i < B; ++i) {
    double s = c[i];
    for (int k = 0; k < i; ++k) s -= L[i][k] * z[k];
    z[i] = s / L[i][i];
  }
  for (int i = B - 1; i >= 0; --i) {
    double s = z[i];
    for (int k = i + 1; k < B; ++k) s -= L[k][i] * beta[k];
    beta[i] = s / L[i][i];
  }
  return 0;
}

/* ---- near ties and reversed decisions (test hook) ------------------------ */
/* An exercise decision (payoff h against fitted continuation value c, both   */
/* at the decision's date) is a near tie when |h - c| <= tie_rel max(|c|, h):  */
/* another correct rounding of the same arithmetic may decide it the other    */
/* way.  Decisions are keyed n P + p (regression paths) and, in the pricing   */
/* pass of the out-of-sample estimator, ORC_KEY_PRICING | (n P + p).  A      */
/* decision whose key is in ctl->flips is taken the other way; everything     */
/* downstream of it (cash flows, earlier regressions) follows.  With no      */
/* control the functions are the plain method.                               */
static int orc_key_in(const uint64_t* keys, uint32_t n, uint64_t key) {
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    const uint32_t mid = lo + (hi - lo) / 2;
    if (keys[mid] == key) return 1;
    if (keys[mid] < key) lo = mid + 1; else hi = mid;
  }
  return 0;
}

/* the decision h > c under the control: near ties recorded, listed
 * decisions reversed */
static int orc_decide(orc_tie_ctl* ctl, uint64_t key, double h, double cont) {
  int ex = h > cont;
  if (!ctl) return ex;
  if (ctl->tie_rel >= 0.0 && fabs(h - cont) <= ctl->tie_rel * fmax(fabs(cont), h)) {
    if (ctl->ties && ctl->n_ties < ctl->max_ties) ctl->ties[ctl->n_ties] = key;
    ++ctl->n_ties;
  }
  if (ctl->n_flips && orc_key_in(ctl->flips, ctl->n_flips, key)) ex = !ex;
  return ex;
}

static int orc_lsmc_core(const double* S, const double* V, uint32_t P, uint32_t N,
                         double S0, double K, double T, double r, double theta, int type,
                         int style, int basis, double out[4], uint32_t* n_singular,
                         double* beta_out, uint8_t* exercise, orc_tie_ctl* ctl) {
  if (!S || !V || !out || P == 0 || N == 0) return -1;
  if (!(K > 0.0) || !(T > 0.0) || !(theta > 0.0) || !isfinite(r)) return -1;
  if (type != ORC_PUT && type != ORC_CALL) return -1;
  if (style != ORC_AMERICAN && style != ORC_EUROPEAN) return -1;
  if (basis != ORC_BASIS_S2 && basis != ORC_BASIS_SV2) return -1;
  const double dt = T / (double)N;
  const double D = exp(-r * dt); /* one-step discount factor */
  double* Y = (double*)malloc(sizeof(double) * P);
  if (!Y) return -2;
  uint32_t singular = 0;
  if (beta_out)
    for (size_t i = 0; i < (size_t)N * 6; ++i) beta_out[i] = NAN;
  if (exercise) memset(exercise, 0, (size_t)N * P);

  /* cash flow at maturity */
  double sum_h = 0.0;
  for (uint32_t p = 0; p < P; ++p) {
    Y[p] = orc_payoff(type, K, S[(size_t)N * P + p]);
    sum_h += Y[p];
  }
  const double european = exp(-r * T) * (sum_h / (double)P);

  if (style == ORC_EUROPEAN) {
    double s = 0.0, s2 = 0.0;
    for (uint32_t p = 0; p < P; ++p) {
      double y = exp(-r * T) * Y[p];
      s += y;
      s2 += y * y;
    }
    double mean = s / (double)P;
    double var = P > 1 ? (s2 - (double)P * mean * mean) / (double)(P - 1) : 0.0;
    out[0] = european;
    out[1] = var > 0.0 ? sqrt(var / (double)P) : 0.0;
    out[2] = european;
    out[3] = european;
    if (n_singular) *n_singular = 0;
    free(Y);
    return 0;
  }

  for (uint32_t n = N - 1; n >= 1; --n) {
    /* discount the cash flow from t_{n+1} to t_n */
    for (uint32_t p = 0; p < P; ++p) Y[p] *= D;
    /* regression of Y on the basis over the in-the-money paths */
    double A[6][6] = {{0}}, c[6] = {0}, beta[6] = {0};
    uint32_t count = 0;
    int B = basis == ORC_BASIS_SV2 ? 6 : 3;
    for (uint32_t p = 0; p < P; ++p) {
      double s = S[(size_t)n * P + p];
      if (!(orc_payoff(type, K, s) > 0.0)) continue;
      double phi[6];
      orc_basis(basis, s, V[(size_t)n * P + p], K, theta, phi);
      for (int i = 0; i < B; ++i) {
        for (int j = 0; j < B; ++j) A[i][j] += phi[i] * phi[j];
        c[i] += phi[i] * Y[p];
      }
      ++count;
    }
    if (count < (uint32_t)B || orc_cholesky_solve(B, A, c, beta) != 0) {
      ++singular;
      continue;
    }
    if (beta_out)
      for (int i = 0; i < 6; ++i) beta_out[(size_t)n * 6 + i] = i < B ? beta[i] : 0.0;
    /* exercise where the payoff beats the fitted continuation value */
    for (uint32_t p = 0; p < P; ++p) {
      double s = S[(size_t)n * P + p];
      double h = orc_payoff(type, K, s);
      if (!(h > 0.0)) continue;
      double phi[6];
      orc_basis(basis, s, V[(size_t)n * P + p], K, theta, phi);
      double cont = 0.0;
      for (int i = 0; i < B; ++i) cont += beta[i] * phi[i];
      if (orc_decide(ctl, (uint64_t)n * P + p, h, cont)) {
        Y[p] = h;
        if (exercise) exercise[(size_t)n * P + p] = 1;
      }
    }
  }
  /* to t_0 */
  double s = 0.0, s2 = 0.0;
  for (uint32_t p = 0; p < P; ++p) {
    double y = D * Y[p];
    s += y;
    s2 += y * y;
  }
  const double mean = s / (double)P;
  const double var = P > 1 ? (s2 - (double)P * mean * mean) / (double)(P - 1) : 0.0;
  const double h0 = orc_payoff(type, K, S0);
  out[0] = h0 > mean ? h0 : mean; /* exercise at t_0 if immediately better */
  out[1] = var > 0.0 ? sqrt(var / (double)P) : 0.0;
  out[2] = european;
  out[3] = mean;
  if (n_singular) *n_singular = singular;
  free(Y);
  return 0;
}

int orc_lsmc(const double* S, const double* V, uint32_t P, uint32_t N,
             double S0, double K, double T, double r, double theta, int type,
             int style, int basis, double out[4], uint32_t* n_singular,
             double* beta_out, uint8_t* exercise) {
  return orc_lsmc_core(S, V, P, N, S0, K, T, r, theta, type, style, basis, out, n_singular,
                       beta_out, exercise, NULL);
}

int orc_lsmc_tie(const double* S, const double* V, uint32_t P, uint32_t N,
                 double S0, double K, double T, double r, double theta, int type,
                 int style, int basis, double out[4], uint32_t* n_singular,
                 orc_tie_ctl* ctl) {
  return orc_lsmc_core(S, V, P, N, S0, K, T, r, theta, type, style, basis, out, n_singular,
                       NULL, NULL, ctl);
}

/* ---- out-of-sample Longstaff-Schwartz ------------------------------------ */
/* The exercise policy estimated by the regressions on one path set (A) is   */
/* applied to an independent path set (B): a path of B stops at the first    */
/* date n in 1..N-1 where it is in the money and its payoff beats the fitted */
/* continuation value beta_n(A) . phi(S_n, v_n), else at N; the estimator is */
/* the mean discounted cash flow (a low-biased price).  Discounting repeats  */
/* the one-step factor as orc_lsmc does, so with B = A the result is the     */
/* in-sample price exactly.                                                  */
static int orc_lsmc_oos_core(const double* SA, const double* VA, const double* SB,
                             const double* VB, uint32_t P, uint32_t N, double S0, double K,
                             double T, double r, double theta, int type, int style, int basis,
                             double out[4], uint32_t* n_singular, orc_tie_ctl* ctl) {
  if (!SA || !VA || !SB || !VB || !out || P == 0 || N == 0) return -1;
  double* beta = (double*)malloc(sizeof(double) * (size_t)N * 6);
  if (!beta) return -2;
  double ins[4];
  int rc = orc_lsmc_core(SA, VA, P, N, S0, K, T, r, theta, type, style, basis, ins, n_singular,
                         beta, NULL, ctl);
  if (rc) { free(beta); return rc; }
  const double dt = T / (double)N;
  const double D = exp(-r * dt);
  const int B = basis == ORC_BASIS_SV2 ? 6 : 3;
  double s = 0.0, s2 = 0.0, sum_h = 0.0;
  for (uint32_t p = 0; p < P; ++p) {
    const double hN = orc_payoff(type, K, SB[(size_t)N * P + p]);
    sum_h += hN;
    double y = hN;
    uint32_t tau = N;
    if (style == ORC_AMERICAN) {
      for (uint32_t n = 1; n < N; ++n) {
        if (isnan(beta[(size_t)n * 6])) continue;  /* no regression at n: no exercise */
        const double sn = SB[(size_t)n * P + p];
        const double h = orc_payoff(type, K, sn);
        if (!(h > 0.0)) continue;
        double phi[6];
        orc_basis(basis, sn, VB[(size_t)n * P + p], K, theta, phi);
        double cont = 0.0;
        for (int i = 0; i < B; ++i) cont += beta[(size_t)n * 6 + i] * phi[i];
        if (orc_decide(ctl, ORC_KEY_PRICING | ((uint64_t)n * P + p), h, cont)) {
          y = h;
          tau = n;
          break;
        }
      }
    }
    /* discount from t_tau to t_0 one step at a time */
    if (style == ORC_AMERICAN) {
      for (uint32_t n = tau; n >= 2; --n) y *= D;
      y *= D;
    } else {
      y *= exp(-r * T);
    }
    s += y;
    s2 += y * y;
  }
  const double mean = s / (double)P;
  const double var = P > 1 ? (s2 - (double)P * mean * mean) / (double)(P - 1) : 0.0;
  const double h0 = orc_payoff(type, K, S0);
  out[0] = style == ORC_AMERICAN && h0 > mean ? h0 : mean;
  out[1] = var > 0.0 ? sqrt(var / (double)P) : 0.0;
  out[2] = exp(-r * T) * (sum_h / (double)P);
  out[3] = mean;
  free(beta);
  return 0;
}

int orc_lsmc_oos(const double* SA, const double* VA, const double* SB, const double* VB,
                 uint32_t P, uint32_t N, double S0, double K, double T, double r,
                 double theta, int type, int style, int basis, double out[4],
                 uint32_t* n_singular) {
  return orc_lsmc_oos_core(SA, VA, SB, VB, P, N, S0, K, T, r, theta, type, style, basis, out,
                           n_singular, NULL);
}

/* ------------------------------------------------------------------------ */
/* Dual (Andersen-Broadie primal-dual) upper bound of the American price.   */
/* The exercise policy is the one fitted by the regressions on the paths of */
/* `stream`.  Outer paths: the first n_outer paths of the pricing stream     */
/* (stream ^ 0x80000000).  Along outer path p, at every date n = 0..N-1, the */
/* value of continuing and following the policy from n + 1 on,              */
/* Q_n = E_n[Z_tau], Z the payoff discounted to t_0, is estimated by the     */
/* mean over n_inner inner paths started from the outer state (x_n, v_n);   */
/* inner path j draws from counter (j, m, stream ^ 0x40000000, 1 + p N + n) */
/* for its step from date m.  The policy's value process is L_n = Z_n where  */
/* the policy exercises (L_N = Z_N) and Q_n elsewhere; the martingale        */
/* pi_0 = 0, pi_{n+1} = pi_n + L_{n+1} - Q_n (the part of L's change that is */
/* not predictable at n); the bound is the mean over outer paths of         */
/* max_{n = 0..N} (Z_n - pi_n), which no stopping rule can beat in          */
/* expectation.                                                              */
/* ------------------------------------------------------------------------ */
/* the payoff h discounted from date n to t_0 by n one-step factors D, as   */
/* orc_lsmc_oos does it */
static double orc_disc(double h, uint32_t n, double D) {
  for (uint32_t i = 0; i < n; ++i) h *= D;
  return h;
}

/* 1 where the policy with date-n coefficients beta_n (NaN: no regression)  */
/* exercises at spot s, stored variance v; *h = the payoff                  */
static int orc_policy_exercises(int type, int basis, double K, double theta,
                                const double* beta_n, double s, double v, double* h) {
  *h = orc_payoff(type, K, s);
  if (isnan(beta_n[0]) || !(*h > 0.0)) return 0;
  double phi[6];
  const int B = orc_basis(basis, s, v, K, theta, phi);
  double cont = 0.0;
  for (int i = 0; i < B; ++i) cont += beta_n[i] * phi[i];
  return *h > cont;
}

/* one step of the scheme from (x, v); *vs = the stored variance (max(v, 0)
 * under full truncation) */
static void orc_step(const orc_heston* m, double dt, int scheme, const double d[3], double* x,
                     double* v, double* vs) {
  if (scheme == ORC_QE) {
    double o[2];
    orc_qe_step(m, dt, *x, *v, d[0], d[1], d[2], o);
    *x = o[0]; *v = o[1]; *vs = o[1];
  } else {
    double o[3];
    orc_ft_step(m, dt, *x, *v, d[1], d[2], o);
    *x = o[0]; *v = o[1]; *vs = o[2];
  }
}

typedef struct {
  const orc_heston* m;
  double T, dt, D;
  int type, scheme, grid, basis;
  uint32_t N, n_strikes, n_inner, n_outer;
  uint64_t seed;
  uint32_t stream;
  const double* strikes;
  const double* beta;  /* n_strikes x N x 6 */
  double* dmax;        /* n_strikes x n_outer: max_n (Z_n - pi_n) */
  double* piN;         /* n_strikes x n_outer: pi_N */
  int rc;
} orc_dual_ctx;

static void orc_dual_path(void* vctx, uint32_t p) {
  orc_dual_ctx* c = (orc_dual_ctx*)vctx;
  const uint32_t N = c->N, nk = c->n_strikes;
  const double theta = c->m->theta, S0 = c->m->S0;
  double* xs = (double*)malloc(sizeof(double) * (N + 1));
  double* vs = (double*)malloc(sizeof(double) * (N + 1));   /* state */
  double* vb = (double*)malloc(sizeof(double) * (N + 1));   /* stored */
  double* Q = (double*)malloc(sizeof(double) * (size_t)nk * N);
  double* z = (double*)malloc(sizeof(double) * nk);
  int* done = (int*)malloc(sizeof(int) * nk);
  if (!xs || !vs || !vb || !Q || !z || !done) {
    c->rc = -2;
    free(xs); free(vs); free(vb); free(Q); free(z); free(done);
    return;
  }
  /* the outer path: pricing stream, path p */
  xs[0] = 0.0; vs[0] = c->m->v0; vb[0] = c->m->v0;
  for (uint32_t n = 0; n < N; ++n) {
    double d[3], x = xs[n], v = vs[n], w;
    orc_draws(c->seed, c->stream ^ 0x80000000u, p, n, c->grid, d);
    orc_step(c->m, c->dt, c->scheme, d, &x, &v, &w);
    xs[n + 1] = x; vs[n + 1] = v; vb[n + 1] = w;
  }
  /* inner estimates Q_n for every date and strike */
  for (uint32_t n = 0; n < N; ++n) {
    for (uint32_t k = 0; k < nk; ++k) Q[(size_t)k * N + n] = 0.0;
    for (uint32_t j = 0; j < c->n_inner; ++j) {
      double x = xs[n], v = vs[n];
      uint32_t left = nk;
      for (uint32_t k = 0; k < nk; ++k) done[k] = 0;
      for (uint32_t m = n; m < N && left > 0; ++m) {
        double d[3], w;
        orc_draws_asset(c->seed, c->stream ^ 0x40000000u, j, m, 1u + p * N + n, c->grid, d);
        orc_step(c->m, c->dt, c->scheme, d, &x, &v, &w);
        const double s = S0 * exp(x);
        const uint32_t date = m + 1;
        for (uint32_t k = 0; k < nk; ++k) {
          if (done[k]) continue;
          double h;
          if (date < N) {
            if (!orc_policy_exercises(c->type, c->basis, c->strikes[k], theta,
                                      c->beta + ((size_t)k * N + date) * 6, s, w, &h))
              continue;
          } else {
            h = orc_payoff(c->type, c->strikes[k], s);
          }
          z[k] = orc_disc(h, date, c->D);
          done[k] = 1;
          --left;
        }
      }
      for (uint32_t k = 0; k < nk; ++k) Q[(size_t)k * N + n] += z[k];
    }
    for (uint32_t k = 0; k < nk; ++k) Q[(size_t)k * N + n] /= (double)c->n_inner;
  }
  /* the martingale and the pathwise maximum, per strike */
  for (uint32_t k = 0; k < nk; ++k) {
    const double K = c->strikes[k];
    double pi = 0.0;
    double best = orc_payoff(c->type, K, S0);  /* n = 0: Z_0 - pi_0 */
    for (uint32_t n = 0; n < N; ++n) {
      const uint32_t date = n + 1;
      const double s = S0 * exp(xs[date]);
      double h, L;
      if (date < N) {
        const int ex = orc_policy_exercises(c->type, c->basis, K, theta,
                                            c->beta + ((size_t)k * N + date) * 6, s, vb[date], &h);
        L = ex ? orc_disc(h, date, c->D) : Q[(size_t)k * N + date];
      } else {
        h = orc_payoff(c->type, K, s);
        L = orc_disc(h, N, c->D);
      }
      pi += L - Q[(size_t)k * N + n];
      const double Z = orc_disc(h, date, c->D);
      if (Z - pi > best) best = Z - pi;
    }
    c->dmax[(size_t)k * c->n_outer + p] = best;
    c->piN[(size_t)k * c->n_outer + p] = pi;
  }
  free(xs); free(vs); free(vb); free(Q); free(z); free(done);
}

int orc_dual_bound(const orc_heston* m, int type, double T, const double* strikes,
                   uint32_t n_strikes, uint32_t P, uint32_t N, int scheme, int grid, int basis,
                   uint64_t seed, uint32_t stream, uint32_t n_outer, uint32_t n_inner,
                   int n_threads, double* out) {
  if (!m || !strikes || !out || n_strikes == 0 || P == 0 || N == 0 || n_outer == 0 ||
      n_inner == 0 || n_outer > P)
    return -1;
  if (!orc_model_ok(m, T, scheme)) return -1;
  if ((uint64_t)n_outer * N + 1 > 0xffffffffull) return -1;
  const size_t cells = (size_t)(N + 1) * P;
  double* SA = (double*)malloc(sizeof(double) * cells);
  double* VA = (double*)malloc(sizeof(double) * cells);
  double* SB = (double*)malloc(sizeof(double) * cells);
  double* VB = (double*)malloc(sizeof(double) * cells);
  double* beta = (double*)malloc(sizeof(double) * (size_t)n_strikes * N * 6);
  double* dmax = (double*)malloc(sizeof(double) * (size_t)n_strikes * n_outer);
  double* piN = (double*)malloc(sizeof(double) * (size_t)n_strikes * n_outer);
  int rc = 0;
  if (!SA || !VA || !SB || !VB || !beta || !dmax || !piN) { rc = -2; goto done; }
  rc = orc_paths(m, T, scheme, grid, P, N, seed, stream, SA, VA, n_threads);
  if (!rc) rc = orc_paths(m, T, scheme, grid, P, N, seed, stream ^ 0x80000000u, SB, VB, n_threads);
  for (uint32_t k = 0; k < n_strikes && !rc; ++k) {
    double ins[4], oos[4];
    uint32_t ns = 0;
    rc = orc_lsmc(SA, VA, P, N, m->S0, strikes[k], T, m->r, m->theta, type, ORC_AMERICAN,
                  basis, ins, &ns, beta + (size_t)k * N * 6, NULL);
    if (!rc)
      rc = orc_lsmc_oos(SA, VA, SB, VB, P, N, m->S0, strikes[k], T, m->r, m->theta, type,
                        ORC_AMERICAN, basis, oos, &ns);
    out[(size_t)k * 6 + 0] = oos[0];
    out[(size_t)k * 6 + 1] = oos[1];
  }
  if (rc) goto done;
  {
    orc_dual_ctx c = {m, T, T / (double)N, exp(-m->r * (T / (double)N)), type, scheme, grid,
                      basis, N, n_strikes, n_inner, n_outer, seed, stream, strikes, beta,
                      dmax, piN, 0};
    orc_parallel_for(n_outer, n_threads, orc_dual_path, &c);
    rc = c.rc;
    for (uint32_t k = 0; k < n_strikes && !rc; ++k) {
      double s = 0.0, s2 = 0.0, t = 0.0, t2 = 0.0;
      for (uint32_t p = 0; p < n_outer; ++p) {
        const double d = dmax[(size_t)k * n_outer + p], q = piN[(size_t)k * n_outer + p];
        s += d; s2 += d * d; t += q; t2 += q * q;
      }
      const double n = (double)n_outer;
      const double mean = s / n, mq = t / n;
      const double var = n_outer > 1 ? (s2 - n * mean * mean) / (n - 1.0) : 0.0;
      const double vq = n_outer > 1 ? (t2 - n * mq * mq) / (n - 1.0) : 0.0;
      out[(size_t)k * 6 + 2] = mean;
      out[(size_t)k * 6 + 3] = var > 0.0 ? sqrt(var / n) : 0.0;
      out[(size_t)k * 6 + 4] = mq;
      out[(size_t)k * 6 + 5] = vq > 0.0 ? sqrt(vq / n) : 0.0;
    }
  }
done:
  free(SA); free(VA); free(SB); free(VB); free(beta); free(dmax); free(piN);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Bump-and-revalue scenarios (the paper gives no Greek method; the Greeks  */
/* are central finite differences under common random numbers: every       */
/* scenario re-simulates with the same counters).                           */
/* Order: base, S+, S-, S+ (gamma), S- (gamma), v0+, v0-, r+, r-, T-, T+.   */
/* ------------------------------------------------------------------------ */
int orc_scenarios(const orc_heston* m, double T, const orc_bumps* b,
                  orc_heston* models, double* Ts, int* kinds) {
  if (!m || !b || !models || !Ts || !kinds) return -1;
  const uint32_t mask = b->greek_mask;
  if (mask & ~31u) return -1;
  const int want_delta = (mask & ORC_GREEK_DELTA) != 0;
  const int want_gamma = (mask & ORC_GREEK_GAMMA) != 0;
  const int gamma_shares = (b->rel_dS_gamma == 0.0 || b->rel_dS_gamma == b->rel_dS);
  int n = 0;
#define ORC_ADD(kind_, model_, T_) \
  do { models[n] = (model_); Ts[n] = (T_); kinds[n] = (kind_); ++n; } while (0)
  ORC_ADD(ORC_SC_BASE, *m, T);
  if (want_delta || (want_gamma && gamma_shares)) {
    if (!(b->rel_dS > 0.0 && b->rel_dS < 1.0)) return -1;
    orc_heston up = *m, dn = *m;
    up.S0 = m->S0 * (1.0 + b->rel_dS);
    dn.S0 = m->S0 * (1.0 - b->rel_dS);
    ORC_ADD(ORC_SC_S_UP, up, T);
    ORC_ADD(ORC_SC_S_DN, dn, T);
  }
  if (want_gamma && !gamma_shares) {
    if (!(b->rel_dS_gamma > 0.0 && b->rel_dS_gamma < 1.0)) return -1;
    orc_heston up = *m, dn = *m;
    up.S0 = m->S0 * (1.0 + b->rel_dS_gamma);
    dn.S0 = m->S0 * (1.0 - b->rel_dS_gamma);
    ORC_ADD(ORC_SC_SG_UP, up, T);
    ORC_ADD(ORC_SC_SG_DN, dn, T);
  }
  if (mask & ORC_GREEK_VEGA) {
    if (!(b->rel_dv0 > 0.0 && b->rel_dv0 < 1.0) || !(m->v0 > 0.0)) return -1;
    orc_heston up = *m, dn = *m;
    up.v0 = m->v0 * (1.0 + b->rel_dv0);
    dn.v0 = m->v0 * (1.0 - b->rel_dv0);
    ORC_ADD(ORC_SC_V_UP, up, T);
    ORC_ADD(ORC_SC_V_DN, dn, T);
  }
  if (mask & ORC_GREEK_RHO) {
    if (!(b->abs_dr > 0.0)) return -1;
    orc_heston up = *m, dn = *m;
    up.r = m->r + b->abs_dr;
    dn.r = m->r - b->abs_dr;
    ORC_ADD(ORC_SC_R_UP, up, T);
    ORC_ADD(ORC_SC_R_DN, dn, T);
  }
  if (mask & ORC_GREEK_THETA) {
    if (!(b->abs_dT > 0.0 && b->abs_dT < T)) return -1;
    ORC_ADD(ORC_SC_T_DN, *m, T - b->abs_dT);
    ORC_ADD(ORC_SC_T_UP, *m, T + b->abs_dT);
  }
#undef ORC_ADD
  return n;
}

typedef struct {
  const double *S, *V, *strikes;
  uint32_t P, N;
  double S0, T, r, theta;
  int type, style, basis;
  double* vals;      /* per strike */
  double* aux;       /* per strike: se, european */
  uint32_t* singular; /* per strike */
  int* rc;
  const double *SB, *VB; /* out of sample: the pricing paths (else NULL) */
} orc_bwd_ctx;

static void orc_bwd_strike(void* vctx, uint32_t k) {
  orc_bwd_ctx* c = (orc_bwd_ctx*)vctx;
  double out[4];
  uint32_t ns = 0;
  int rc = c->SB ? orc_lsmc_oos(c->S, c->V, c->SB, c->VB, c->P, c->N, c->S0, c->strikes[k],
                                c->T, c->r, c->theta, c->type, c->style, c->basis, out, &ns)
                 : orc_lsmc(c->S, c->V, c->P, c->N, c->S0, c->strikes[k], c->T, c->r,
                            c->theta, c->type, c->style, c->basis, out, &ns, NULL, NULL);
  c->rc[k] = rc;
  c->vals[k] = out[0];
  c->aux[2 * k] = out[1];
  c->aux[2 * k + 1] = out[2];
  c->singular[k] = ns;
}

/* Central differences of the revaluations (Greeks per Sec. 2.2's purpose;
 * the bump readings of orc_scenarios): delta from the S pair, gamma from its
 * own S pair or the delta pair with the base, vega per unit of v0, rho per
 * unit rate, theta = -dV/dT from the T pair.  vals[s] is the price of
 * scenario s of kinds[]. */
void orc_greeks_from_values(const orc_heston* m, const orc_bumps* b, const int* kinds,
                            const double* vals, int n_sc, orc_result* o) {
  double v[ORC_SC_COUNT];
  int have[ORC_SC_COUNT] = {0};
  for (int s = 0; s < n_sc; ++s) {
    v[kinds[s]] = vals[s];
    have[kinds[s]] = 1;
  }
  memset(o, 0, sizeof(*o));
  o->price = v[ORC_SC_BASE];
  o->price_se = o->european_price = NAN;
  o->delta = o->gamma = o->vega = o->rho = o->theta = NAN;
  const double S0 = m->S0;
  if ((b->greek_mask & ORC_GREEK_DELTA) && have[ORC_SC_S_UP])
    o->delta = (v[ORC_SC_S_UP] - v[ORC_SC_S_DN]) / (2.0 * b->rel_dS * S0);
  if (b->greek_mask & ORC_GREEK_GAMMA) {
    if (have[ORC_SC_SG_UP]) {
      double h = b->rel_dS_gamma * S0;
      o->gamma = (v[ORC_SC_SG_UP] - 2.0 * v[ORC_SC_BASE] + v[ORC_SC_SG_DN]) / (h * h);
    } else {
      double h = b->rel_dS * S0;
      o->gamma = (v[ORC_SC_S_UP] - 2.0 * v[ORC_SC_BASE] + v[ORC_SC_S_DN]) / (h * h);
    }
  }
  if (b->greek_mask & ORC_GREEK_VEGA)
    o->vega = (v[ORC_SC_V_UP] - v[ORC_SC_V_DN]) / (2.0 * b->rel_dv0 * m->v0);
  if (b->greek_mask & ORC_GREEK_RHO)
    o->rho = (v[ORC_SC_R_UP] - v[ORC_SC_R_DN]) / (2.0 * b->abs_dr);
  if (b->greek_mask & ORC_GREEK_THETA)
    o->theta = (v[ORC_SC_T_DN] - v[ORC_SC_T_UP]) / (2.0 * b->abs_dT);
  o->n_revaluations = (uint32_t)n_sc;
}

int orc_price_greeks(const orc_heston* m, int type, int style, double T,
                     const double* strikes, uint32_t n_strikes, uint32_t P,
                     uint32_t N, int scheme, int grid, int basis,
                     const orc_bumps* b, uint64_t seed, uint32_t stream,
                     int n_threads, orc_result* out, double* scen_prices) {
  return orc_price_greeks_ex(m, type, style, T, strikes, n_strikes, P, N, scheme, grid, basis,
                             b, seed, stream, 0, 0, n_threads, out, scen_prices);
}

/* Paths of scenario s as a 16-bit path store holds them (store = 1:
 * binary16, 2: bfloat16).  A stored value is exp(x) of the simulation (x =
 * log(S / S0), started at 0) or its variance, rounded to the format; a
 * scenario reads S = S0 exp(x) as its S0 times the stored value.  A rate
 * bump moves every log-price of the scheme by (+-dr) t_n and nothing else,
 * so the rate scenarios read the base simulation's stored values times
 * exp(+-dr t_n). */
static int orc_paths_store16(const orc_heston* base, const orc_heston* ms, int kind,
                             double T, int scheme, int grid, uint32_t P, uint32_t N,
                             uint64_t seed, uint32_t stream, int store, double* S,
                             double* V, int n_threads) {
  const int rate = kind == ORC_SC_R_UP || kind == ORC_SC_R_DN;
  orc_heston unit = rate ? *base : *ms;
  unit.S0 = 1.0;  /* rows of exp(x) */
  const int rc = orc_paths(&unit, T, scheme, grid, P, N, seed, stream, S, V, n_threads);
  if (rc) return rc;
  const double dr = rate ? ms->r - base->r : 0.0;
  const double dt = T / (double)N;
  for (uint32_t n = 0; n <= N; ++n) {
    const double f = rate ? ms->S0 * exp((double)n * dr * dt) : ms->S0;
    for (uint32_t p = 0; p < P; ++p) {
      const size_t i = (size_t)n * P + p;
      const double e = store == 1 ? orc_round_f16(S[i]) : orc_round_bf16(S[i]);
      S[i] = f * e;
      V[i] = store == 1 ? orc_round_f16(V[i]) : orc_round_bf16(V[i]);
    }
  }
  return 0;
}

int orc_price_greeks_ex(const orc_heston* m, int type, int style, double T,
                        const double* strikes, uint32_t n_strikes, uint32_t P,
                        uint32_t N, int scheme, int grid, int basis,
                        const orc_bumps* b, uint64_t seed, uint32_t stream,
                        int out_of_sample, int store, int n_threads, orc_result* out,
                        double* scen_prices) {
  if (!m || !strikes || !b || !out || n_strikes == 0 || P == 0 || N == 0)
    return -1;
  if (store < 0 || store > 2) return -1;
  orc_heston models[ORC_SC_COUNT];
  double Ts[ORC_SC_COUNT];
  int kinds[ORC_SC_COUNT];
  int n_sc = orc_scenarios(m, T, b, models, Ts, kinds);
  if (n_sc < 1) return -1;
  for (int s = 0; s < n_sc; ++s)
    if (!orc_model_ok(&models[s], Ts[s], scheme)) return -1;
  for (uint32_t k = 0; k < n_strikes; ++k)
    if (!(strikes[k] > 0.0) || !isfinite(strikes[k])) return -1;

  size_t cells = (size_t)(N + 1) * P;
  double* S = (double*)malloc(sizeof(double) * cells);
  double* V = (double*)malloc(sizeof(double) * cells);
  /* out of sample: pricing paths from stream ^ 0x80000000 */
  double* SB = out_of_sample ? (double*)malloc(sizeof(double) * cells) : NULL;
  double* VB = out_of_sample ? (double*)malloc(sizeof(double) * cells) : NULL;
  double* vals = (double*)malloc(sizeof(double) * n_sc * n_strikes);
  double* aux = (double*)malloc(sizeof(double) * 2 * n_strikes);
  uint32_t* sing = (uint32_t*)calloc((size_t)n_sc * n_strikes, sizeof(uint32_t));
  int* rcs = (int*)malloc(sizeof(int) * n_strikes);
  double* base_aux = (double*)malloc(sizeof(double) * 2 * n_strikes);
  int rc = 0;
  if (!S || !V || !vals || !aux || !sing || !rcs || !base_aux ||
      (out_of_sample && (!SB || !VB))) { rc = -2; goto done; }

  for (int s = 0; s < n_sc && rc == 0; ++s) {
    if (store)
      rc = orc_paths_store16(&models[0], &models[s], kinds[s], Ts[s], scheme, grid, P, N,
                             seed, stream, store, S, V, n_threads);
    else
      rc = orc_paths(&models[s], Ts[s], scheme, grid, P, N, seed, stream, S, V,
                     n_threads);
    if (rc) break;
    if (out_of_sample) {
      if (store)
        rc = orc_paths_store16(&models[0], &models[s], kinds[s], Ts[s], scheme, grid, P, N,
                               seed, stream ^ 0x80000000u, store, SB, VB, n_threads);
      else
        rc = orc_paths(&models[s], Ts[s], scheme, grid, P, N, seed, stream ^ 0x80000000u, SB,
                       VB, n_threads);
      if (rc) break;
    }
    orc_bwd_ctx c = {S, V, strikes, P, N, models[s].S0, Ts[s], models[s].r,
                     models[s].theta, type, style, basis,
                     vals + (size_t)s * n_strikes, aux,
                     sing + (size_t)s * n_strikes, rcs, SB, VB};
    orc_parallel_for(n_strikes, n_threads, orc_bwd_strike, &c);
    for (uint32_t k = 0; k < n_strikes; ++k)
      if (rcs[k]) rc = rcs[k];
    if (s == 0) memcpy(base_aux, aux, sizeof(double) * 2 * n_strikes);
  }
  if (rc) goto done;

  for (uint32_t k = 0; k < n_strikes; ++k) {
    double v[ORC_SC_COUNT];
    uint32_t ns = 0;
    for (int s = 0; s < n_sc; ++s) {
      v[s] = vals[(size_t)s * n_strikes + k];
      ns += sing[(size_t)s * n_strikes + k];
    }
    orc_result* o = &out[k];
    orc_greeks_from_values(m, b, kinds, v, n_sc, o);
    o->price_se = base_aux[2 * k];
    o->european_price = base_aux[2 * k + 1];
    o->n_singular = ns;
    o->status = ns ? 1 : 0;
  }
  if (scen_prices) memcpy(scen_prices, vals, sizeof(double) * n_sc * n_strikes);
done:
  free(S); free(V); free(vals); free(aux); free(sing); free(rcs); free(base_aux);
  free(SB); free(VB);
  return rc;
}

/* ---- one revaluation under reversed near-tie decisions (test hook) ------ */
typedef struct {
  const double *S, *V, *SB, *VB;
  uint32_t P, N;
  double S0, K, T, r, theta;
  int type, style, basis;
  const uint64_t* keys;
  uint32_t n_keys;
  double* out;
  int* rcs;
} orc_alt_ctx;

static void orc_alt_one(void* vctx, uint32_t set) {
  const orc_alt_ctx* c = (const orc_alt_ctx*)vctx;
  uint64_t flips[ORC_MAX_ALT_KEYS];
  uint32_t nf = 0;
  for (uint32_t i = 0; i < c->n_keys; ++i)
    if (set & (1u << i)) flips[nf++] = c->keys[i];
  orc_tie_ctl ctl = {-1.0, NULL, 0, 0, flips, nf};
  double o[4];
  uint32_t ns = 0;
  c->rcs[set] = c->SB ? orc_lsmc_oos_core(c->S, c->V, c->SB, c->VB, c->P, c->N, c->S0, c->K,
                                          c->T, c->r, c->theta, c->type, c->style, c->basis,
                                          o, &ns, &ctl)
                      : orc_lsmc_core(c->S, c->V, c->P, c->N, c->S0, c->K, c->T, c->r,
                                      c->theta, c->type, c->style, c->basis, o, &ns, NULL,
                                      NULL, &ctl);
  c->out[set] = o[0];
}

static int orc_cmp_u64(const void* a, const void* b) {
  const uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
  return x < y ? -1 : x > y;
}

int orc_scenario_alternatives(const orc_heston* m, int type, int style, double T, double K,
                              uint32_t P, uint32_t N, int scheme, int grid, int basis,
                              const orc_bumps* b, uint64_t seed, uint32_t stream,
                              int out_of_sample, int store, int sc, double tie_rel,
                              const uint64_t* keys, uint32_t n_keys, double* out,
                              uint64_t* ties, uint32_t max_ties, uint32_t* n_ties,
                              int n_threads) {
  if (!m || !b || !out || P == 0 || N == 0 || n_keys > ORC_MAX_ALT_KEYS ||
      (n_keys && !keys) || store < 0 || store > 2)
    return -1;
  orc_heston models[ORC_SC_COUNT];
  double Ts[ORC_SC_COUNT];
  int kinds[ORC_SC_COUNT];
  const int n_sc = orc_scenarios(m, T, b, models, Ts, kinds);
  if (n_sc < 1 || sc < 0 || sc >= n_sc) return -1;
  if (!orc_model_ok(&models[sc], Ts[sc], scheme) || !(K > 0.0) || !isfinite(K)) return -1;
  const size_t cells = (size_t)(N + 1) * P;
  double* S = (double*)malloc(sizeof(double) * cells);
  double* V = (double*)malloc(sizeof(double) * cells);
  double* SB = out_of_sample ? (double*)malloc(sizeof(double) * cells) : NULL;
  double* VB = out_of_sample ? (double*)malloc(sizeof(double) * cells) : NULL;
  const uint32_t n_sets = 1u << n_keys;
  int* rcs = (int*)calloc(n_sets, sizeof(int));
  uint64_t* sorted = (uint64_t*)malloc(sizeof(uint64_t) * (n_keys ? n_keys : 1));
  int rc = 0;
  if (!S || !V || !rcs || !sorted || (out_of_sample && (!SB || !VB))) { rc = -2; goto done; }
  /* the revaluation's paths exactly as orc_price_greeks_ex simulates them */
  if (store)
    rc = orc_paths_store16(&models[0], &models[sc], kinds[sc], Ts[sc], scheme, grid, P, N,
                           seed, stream, store, S, V, n_threads);
  else
    rc = orc_paths(&models[sc], Ts[sc], scheme, grid, P, N, seed, stream, S, V, n_threads);
  if (rc == 0 && out_of_sample) {
    if (store)
      rc = orc_paths_store16(&models[0], &models[sc], kinds[sc], Ts[sc], scheme, grid, P, N,
                             seed, stream ^ 0x80000000u, store, SB, VB, n_threads);
    else
      rc = orc_paths(&models[sc], Ts[sc], scheme, grid, P, N, seed, stream ^ 0x80000000u, SB,
                     VB, n_threads);
  }
  if (rc) goto done;
  if (n_ties) {
    /* the near ties of the plain run */
    orc_tie_ctl ctl = {tie_rel, ties, ties ? max_ties : 0, 0, NULL, 0};
    double o[4];
    uint32_t ns = 0;
    rc = out_of_sample
             ? orc_lsmc_oos_core(S, V, SB, VB, P, N, models[sc].S0, K, Ts[sc], models[sc].r,
                                 models[sc].theta, type, style, basis, o, &ns, &ctl)
             : orc_lsmc_core(S, V, P, N, models[sc].S0, K, Ts[sc], models[sc].r,
                             models[sc].theta, type, style, basis, o, &ns, NULL, NULL, &ctl);
    *n_ties = ctl.n_ties;
    if (rc) goto done;
  }
  for (uint32_t i = 0; i < n_keys; ++i) sorted[i] = keys[i];
  qsort(sorted, n_keys, sizeof(uint64_t), orc_cmp_u64);
  {
    /* every subset of the keys reversed (orc_alt_one takes them in sorted
       order, so bit i of a subset is the i-th smallest key) */
    orc_alt_ctx c = {S, V, SB, VB, P, N, models[sc].S0, K, Ts[sc], models[sc].r,
                     models[sc].theta, type, style, basis, sorted, n_keys, out, rcs};
    orc_parallel_for(n_sets, n_threads, orc_alt_one, &c);
    for (uint32_t i = 0; i < n_sets; ++i)
      if (rcs[i]) rc = rcs[i];
  }
done:
  free(S); free(V); free(SB); free(VB); free(rcs); free(sorted);
  return rc;
}

/* ---- array forms of the scalar functions (loops only, for the tests) --- */
void orc_philox_n(const uint32_t* ctr, const uint32_t key[2], uint32_t* out,
                  size_t n) {
  for (size_t i = 0; i < n; ++i) orc_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

void orc_norm_inv_n(const double* u, double* z, size_t n) {
  for (size_t i = 0; i < n; ++i) z[i] = orc_norm_inv(u[i]);
}

void orc_draws_n(uint64_t seed, uint32_t stream, const uint32_t* path,
                 const uint32_t* step, size_t n, int grid, double* out) {
  for (size_t i = 0; i < n; ++i)
    orc_draws(seed, stream, path[i], step[i], grid, out + 3 * i);
}
