// heston_step.cuh -- one time step of the Heston model in each working
// precision: Andersen's quadratic-exponential scheme (the paper's
// discretisation, Sec. 2.2.1) and full-truncation Euler, with the per-group
// scheme constants.  Shared by the forward pass (forward.cu) and the inner
// simulations of the dual upper bound (dual.cu).
#pragma once

#include <type_traits>

#include "device_common.cuh"
#include "df_math.cuh"
#include "dfloat.cuh"
#include "plan.h"

namespace lsmc {

// Elementary functions per precision; the float-pair ones read their
// tables from shared memory (t), the others ignore it.
template <typename Real> struct Fm;
template <> struct Fm<double> {
  __device__ static double div(double a, double b) { return a / b; }
  __device__ static double sqrt_(double a) { return sqrt(a); }
  __device__ static double log_(double a, const DfTables*) { return log_f64(a); }
  __device__ static double exp_(double a, const DfTables*) { return exp_f64(a); }
};
template <> struct Fm<float> {
  __device__ static float div(float a, float b) { return __fdividef(a, b); }
  __device__ static float sqrt_(float a) {
    float r;  // approximate square root (MUFU), exact at 0
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
  }
  __device__ static float log_(float a, const DfTables*) { return __logf(a); }
  __device__ static float exp_(float a, const DfTables*) { return __expf(a); }
};
template <> struct Fm<df> {
  __device__ static df div(df a, df b) { return a / b; }
  __device__ static df sqrt_(df a) { return sqrt_df(a); }
  __device__ static df log_(df a, const DfTables* t) { return log_df(a, t->exp2); }
  __device__ static df exp_(df a, const DfTables* t) { return exp_df(a, t->exp2); }
};

template <typename Real>
struct GroupConst {
  // QE: m = mA + mB v, s^2 = sA + sB v, x1 = x + c0 + K1 v + K2 v1 + sqrt(K3 (v + v1)) Z
  Real mA, mB, sA, sB, c0, K1, K2, K3;
  // FT-Euler
  Real dt, kdt, theta, xi, rho, rhob, mudt;
  Real v0, out_scale;
  void* E;            // rows of the path store (element type: the launch's store format)
  void* V;
  Real* CX;
  Real* CV;
  uint64_t ld;
};

// Scheme constants of one path group, from the model (Andersen 2008 for QE
// with gamma1 = gamma2 = 1/2; the plain Euler coefficients for FT).
template <typename Real>
__device__ void make_group_const(const FwdGroup& g, GroupConst<Real>& c) {
  const double dt = g.dt, k = g.kappa, th = g.theta, xi = g.xi, rho = g.rho;
  const double E = exp(-k * dt);
  const double omE = -expm1(-k * dt);  // 1 - E without cancellation
  c.mA = (Real)(th * omE);
  c.mB = (Real)E;
  if (xi > 0.0) {
    c.sB = (Real)(xi * xi * E * omE / k);
    c.sA = (Real)(th * xi * xi * omE * omE / (2.0 * k));
    const double K0 = -rho * k * th * dt / xi;
    const double h = 0.5 * dt * (k * rho / xi - 0.5);
    c.K1 = (Real)(h - rho / xi);
    c.K2 = (Real)(h + rho / xi);
    c.c0 = (Real)((g.r - g.q) * dt + K0);
  } else {
    c.sA = c.sB = c.K1 = c.K2 = c.c0 = (Real)0;
  }
  c.K3 = (Real)(0.5 * dt * (1.0 - rho * rho));
  c.dt = (Real)dt;
  c.kdt = (Real)(k * dt);
  c.theta = (Real)th;
  c.xi = (Real)xi;
  c.rho = (Real)rho;
  c.rhob = (Real)sqrt(1.0 - rho * rho);
  c.mudt = (Real)((g.r - g.q) * dt);
  c.v0 = (Real)g.v0;
  c.out_scale = (Real)g.out_scale;
  c.E = g.E;
  c.V = g.V;
  c.CX = (Real*)g.CX;
  c.CV = (Real*)g.CV;
  c.ld = g.ld;
}

// Andersen QE step: variance by the quadratic branch (psi <= 1.5) or the
// exponential branch, then the log price from both variances.  With
// psi = s^2 / m^2 the branch quantities are written with one division
// each: 2 / psi = 2 m^2 / s^2, p = (psi - 1) / (psi + 1) = (s^2 - m^2) /
// (s^2 + m^2), 1 - p = 2 m^2 / (s^2 + m^2), 1 / beta = m / (1 - p); the
// point mass is taken when U_V <= p, i.e. 1 - U_V >= 1 - p.
template <typename Real>
__device__ __forceinline__ void qe_core(Real mA, Real mB, Real sA, Real sB, Real c0, Real K1,
                                        Real K2, Real K3, Real& x, Real& v, Real omu, Real zV,
                                        Real zX, const DfTables* t) {
  using F = Fm<Real>;
  const Real m = fma(mB, v, mA);
  const Real s2 = fma(sB, v, sA);
  const Real m2 = m * m;
  Real v1;
  if (s2 <= (Real)1.5 * m2) {
    const Real inv = F::div(m2 + m2, s2);
    const Real tt = inv - (Real)1;
    const Real b2 = tt + F::sqrt_(inv * tt);
    const Real b = F::sqrt_(b2);
    const Real a = F::div(m, (Real)1 + b2);
    const Real q = b + zV;
    v1 = a * q * q;
  } else {
    const Real rden = F::div((Real)1, s2 + m2);
    const Real omp = (m2 + m2) * rden;
    v1 = (omu >= omp) ? (Real)0 : F::div(m, omp) * F::log_(F::div(omp, omu), t);
  }
  x = x + c0 + K1 * v + K2 * v1 + F::sqrt_(K3 * (v + v1)) * zX;
  v = v1;
}

template <typename Real>
__device__ __forceinline__ void qe_step(const GroupConst<Real>& c, Real& x, Real& v,
                                        Real omu, Real zV, Real zX, const DfTables* t) {
  qe_core<Real>(c.mA, c.mB, c.sA, c.sB, c.c0, c.K1, c.K2, c.K3, x, v, omu, zV, zX, t);
}

// Full-truncation Euler: v+ = max(v, 0) in drift and diffusion.
template <typename Real>
__device__ __forceinline__ void ft_step(const GroupConst<Real>& c, Real& x,
                                        Real& v, Real zV, Real zX) {
  using F = Fm<Real>;
  const Real vp = v > (Real)0 ? v : (Real)0;
  const Real sq = F::sqrt_(vp * c.dt);
  const Real v1 = v + c.kdt * (c.theta - vp) + c.xi * sq * zV;
  x = x + (c.mudt - (Real)0.5 * vp * c.dt) + sq * (c.rho * zV + c.rhob * zX);
  v = v1;
}

}  // namespace lsmc
