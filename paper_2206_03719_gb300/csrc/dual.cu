// dual.cu -- dual (Andersen-Broadie primal-dual) upper bound of the American
// price for the strikes of one request.
//
// The Longstaff-Schwartz policy (the regressions' coefficients of every date,
// cash flows discounted to t_0) defines a stopping rule and its value
// process L: L_n is the discounted payoff Z_n where the rule exercises
// (always at maturity) and the value of continuing, Q_n = E_n[Z_tau] with tau
// the rule's next exercise date, elsewhere.  The martingale part of L,
// pi_0 = 0, pi_{n+1} = pi_n + L_{n+1} - Q_n, gives the upper bound
// E[max_n (Z_n - pi_n)] (Andersen and Broadie; the duality of Rogers and of
// Haugh and Kogan), the gap to the policy's own (lower-bound) price measuring
// how far the policy is from optimal.
//
// Outer paths: the first n_outer paths of the pricing stream (stream ^
// 0x80000000), re-simulated here with the forward pass's arithmetic.  Q_n is
// estimated along each outer path at every date by n_inner inner paths
// started from the outer state; inner path j of outer path p started at date
// n draws from Philox counter (j, m, stream ^ 0x40000000, 1 + p N + n) for its
// step from date m.  The inner paths of a (p, n) pair are shared by all the
// request's strikes (each strike follows its own rule on them).
//
// Kernels: outer states (a thread per outer path); inner estimates (a CTA
// per outer path and date, a thread per inner path); the pathwise maximum
// (a thread per outer path and strike); fixed-order sums per strike.
#include "checked.cuh"
#include <type_traits>

#include "device_common.cuh"
#include "df_math.cuh"
#include "dfloat.cuh"
#include "exercise.cuh"
#include "heston_step.cuh"
#include "kernels.h"
#include "plan.h"

namespace lsmc {

namespace {

constexpr int kDualBlock = 128;  // threads (inner paths at a time) per CTA

template <typename Real>
__device__ __forceinline__ bool flag_on(Real f);
template <> __device__ __forceinline__ bool flag_on<double>(double f) {
  return __double_as_longlong(f) != 0;
}
template <> __device__ __forceinline__ bool flag_on<float>(float f) { return __float_as_int(f) != 0; }
template <> __device__ __forceinline__ bool flag_on<df>(df f) { return __float_as_int(f.hi) != 0; }


// The rule of one strike at date n (1..N-1) for a path with row value E
// (S = s_n E) and stored variance v: exercise where the regression was
// solved, the path is in the money and its discounted payoff beats the
// fitted continuation value -- the backward pass's test with the same
// operations, after the same float screen (q).  *z: the discounted cash flow
// of exercising.
template <typename Real, int BASIS>
__device__ __forceinline__ bool rule_exercises(const Real* t, const ScreenConsts& q, int type,
                                               Real K, Real invK, Real invTh, Real E, Real v,
                                               double* z, uint32_t* ties) {
  if (!flag_on(t[6]) || !itm_test(type, K, t[7], E, threshold_bits(t[10]))) return false;
  int pre = 2;
  if constexpr (!std::is_same<Real, float>::value)
    pre = exercise_screen<BASIS>(q, type, approx_float(E),
                                 BASIS == kBasisSV2 ? approx_float(v) : 0.0f);
  if (pre == 0) return false;
  const Real S = t[7] * E;
  const Real h = intrinsic<Real>(type, K, S);
  const Real d1 = t[8], d1lo = t[9];
  const Real hd = qmul(h, d1);
  if (pre == 2) {
    const Real x = qfma(S, invK, (Real)-1);
    Real c = qfma(qfma(t[2], x, t[1]), x, t[0]);
    if (BASIS == kBasisSV2) {
      const Real w = qfma(v, invTh, (Real)-1);
      c = qfma(qfma(t[5], w, qfma(t[4], x, t[3])), w, c);
    }
    bool exercise, tie;
    decide<Real>(hd, c, exercise, tie);
    if (tie) ++*ties;
    if (!exercise) return false;
  }
  Real hz;
  if constexpr (std::is_same<Real, df>::value) hz = quick_two_sum(hd.hi, hd.lo);
  else hz = fma(h, d1, h * d1lo);
  *z = (double)hz;
  return true;
}

// the payoff at S of the maturity date, discounted (row N of the table)
template <typename Real>
__device__ __forceinline__ double maturity_cash(const Real* tN, int type, Real K, Real S) {
  const Real h = payoff<Real>(type, K, S);
  return (double)fma(h, tN[8], h * tN[9]);
}

// the payoff at S of date n < N, discounted as an exercise cash flow
template <typename Real>
__device__ __forceinline__ double date_cash(const Real* t, int type, Real K, Real S) {
  const Real h = payoff<Real>(type, K, S);
  if constexpr (std::is_same<Real, df>::value) {
    const df hd = qmul(h, t[8]);
    return (double)quick_two_sum(hd.hi, hd.lo);
  } else {
    return (double)fma(h, t[8], h * t[9]);
  }
}

template <typename Real>
__device__ __forceinline__ Real stored_variance(int scheme, Real v) {
  return (scheme == kSchemeFT && v < (Real)0) ? (Real)0 : v;
}

}  // namespace

// Outer states x_n, v_n (n = 0..N) of pricing path p (a thread per path),
// with the forward pass's arithmetic.
template <typename Real, int SCHEME>
__global__ void __launch_bounds__(kDualBlock) dual_outer_kernel(DualArgs a) {
  __shared__ GroupConst<Real> gc;
  constexpr bool kPair = std::is_same<Real, df>::value;
  __shared__ __align__(16) unsigned char tab_raw[kPair ? sizeof(DfTables) : 16];
  DfTables* tabs = reinterpret_cast<DfTables*>(tab_raw);
  if (threadIdx.x == 0) make_group_const<Real>(a.group, gc);
  if constexpr (kPair) load_df_tables(tabs);
  __syncthreads();
  const uint32_t p = blockIdx.x * kDualBlock + threadIdx.x;
  if (p >= a.n_outer) return;
  const uint2 key = make_uint2((uint32_t)a.seed, (uint32_t)(a.seed >> 32));
  Real* X = (Real*)a.X;
  Real* V = (Real*)a.V;
  Real x = (Real)0, v = gc.v0;
  CHK_ST(a.chk, &X[p], x);
  CHK_ST(a.chk, &V[p], v);
  for (uint32_t n = 0; n < a.N; ++n) {
    const uint4 w = philox4x32_10(make_uint4(p, n, a.stream ^ 0x80000000u, 0u), key);
    Real u, omu, zV, zX;
    Draw<Real>::make(w, u, omu, zV, zX, tabs);
    if (SCHEME == kSchemeQE) qe_step<Real>(gc, x, v, omu, zV, zX, tabs);
    else ft_step<Real>(gc, x, v, zV, zX);
    CHK_ST(a.chk, &X[(size_t)(n + 1) * a.n_outer + p], x);
    CHK_ST(a.chk, &V[(size_t)(n + 1) * a.n_outer + p], v);
  }
}

// Inner estimates: CTA (p, n) simulates n_inner paths from outer state
// (x_n, v_n) over dates n+1..N, each strike following its rule, and writes
// Q[k][p][n] = the mean discounted cash flow of strike k.
template <typename Real, int SCHEME, int BASIS>
__global__ void __launch_bounds__(kDualBlock) dual_inner_kernel(DualArgs a) {
  __shared__ GroupConst<Real> gc;
  constexpr bool kPair = std::is_same<Real, df>::value;
  __shared__ __align__(16) unsigned char tab_raw[kPair ? sizeof(DfTables) : 16];
  DfTables* tabs = reinterpret_cast<DfTables*>(tab_raw);
  __shared__ double s_acc[kMaxDualStrikes][kDualBlock];
  __shared__ uint32_t s_ties[kDualBlock];
  __shared__ const Real* s_tab[kMaxDualStrikes];
  __shared__ const ScreenConsts* s_scr[kMaxDualStrikes];
  __shared__ Real s_K[kMaxDualStrikes], s_invK[kMaxDualStrikes], s_invTh[kMaxDualStrikes];
  const int tid = threadIdx.x;
  const uint32_t N = a.N, nk = a.n_strikes;
  const uint32_t p = blockIdx.x / N, n = blockIdx.x % N;
  if (tid == 0) make_group_const<Real>(a.group, gc);
  if (tid < (int)nk) {
    const BwdInstance I = CHK_LD(a.chk, &a.inst[a.inst_of_strike[tid]]);
    s_tab[tid] = (const Real*)I.oos_tab;
    s_scr[tid] = (const ScreenConsts*)I.oos_screen;
    s_K[tid] = (Real)I.K;
    s_invK[tid] = (Real)I.invK;
    s_invTh[tid] = (Real)I.inv_theta;
  }
  for (uint32_t k = 0; k < nk; ++k) s_acc[k][tid] = 0.0;
  if constexpr (kPair) load_df_tables(tabs);
  __syncthreads();
  const int type = a.type;
  const uint2 key = make_uint2((uint32_t)a.seed, (uint32_t)(a.seed >> 32));
  const Real x0 = CHK_LD(a.chk, &((const Real*)a.X)[(size_t)n * a.n_outer + p]);
  const Real v0 = CHK_LD(a.chk, &((const Real*)a.V)[(size_t)n * a.n_outer + p]);
  const uint32_t all = nk >= 32 ? 0xffffffffu : (1u << nk) - 1u;
  const uint32_t w3 = 1u + p * N + n;
  uint32_t ties = 0;
  for (uint32_t j = tid; j < a.n_inner; j += kDualBlock) {
    Real x = x0, v = v0;
    uint32_t done = 0;
    for (uint32_t m = n; m < N && done != all; ++m) {
      const uint4 w = philox4x32_10(make_uint4(j, m, a.stream ^ 0x40000000u, w3), key);
      Real u, omu, zV, zX;
      Draw<Real>::make(w, u, omu, zV, zX, tabs);
      if (SCHEME == kSchemeQE) qe_step<Real>(gc, x, v, omu, zV, zX, tabs);
      else ft_step<Real>(gc, x, v, zV, zX);
      const Real E = Fm<Real>::exp_(x, tabs);
      const Real vs = stored_variance<Real>(SCHEME, v);
      const uint32_t date = m + 1;
      for (uint32_t k = 0; k < nk; ++k) {
        if ((done >> k) & 1u) continue;
        const Real* t = s_tab[k] + (size_t)date * kOosConsts;
        if (!CHK_OK(a.chk, t, sizeof(Real) * kOosConsts) ||
            !CHK_OK(a.chk, &s_scr[k][date], sizeof(ScreenConsts))) {
          done |= 1u << k;
          continue;
        }
        if (date < N) {
          double z;
          if (rule_exercises<Real, BASIS>(t, s_scr[k][date], type, s_K[k], s_invK[k],
                                          s_invTh[k], E, vs, &z, &ties)) {
            s_acc[k][tid] += z;
            done |= 1u << k;
          }
        } else {
          s_acc[k][tid] += maturity_cash<Real>(t, type, s_K[k], t[7] * E);
          done |= 1u << k;
        }
      }
    }
  }
  s_ties[tid] = ties;
  __syncthreads();
  // fixed-order sums: thread k adds strike k's column in thread order
  if (tid < (int)nk) {
    double s = 0.0;
    for (int i = 0; i < kDualBlock; ++i) s += s_acc[tid][i];
    CHK_ST(a.chk, &a.Q[((size_t)tid * a.n_outer + p) * N + n], s / (double)a.n_inner);
  }
  if (tid == 0) {
    uint32_t t = 0;
    for (int i = 0; i < kDualBlock; ++i) t += s_ties[i];
    CHK_ST(a.chk, &a.inner_ties[blockIdx.x], t);
  }
}

// Pathwise maximum of Z_n - pi_n for outer path p and strike k = blockIdx.y.
template <typename Real, int SCHEME, int BASIS>
__global__ void __launch_bounds__(kDualBlock) dual_max_kernel(DualArgs a) {
  constexpr bool kPair = std::is_same<Real, df>::value;
  __shared__ __align__(16) unsigned char tab_raw[kPair ? sizeof(DfTables) : 16];
  DfTables* tabs = reinterpret_cast<DfTables*>(tab_raw);
  if constexpr (kPair) load_df_tables(tabs);
  __syncthreads();
  const uint32_t k = blockIdx.y;
  const uint32_t p = blockIdx.x * kDualBlock + threadIdx.x;
  if (p >= a.n_outer) return;
  if (!CHK_OK(a.chk, &a.inst[a.inst_of_strike[k]], sizeof(BwdInstance))) return;
  const BwdInstance& I = a.inst[a.inst_of_strike[k]];
  const Real* tab = (const Real*)I.oos_tab;
  const ScreenConsts* scr = (const ScreenConsts*)I.oos_screen;
  const Real K = (Real)I.K, invK = (Real)I.invK, invTh = (Real)I.inv_theta;
  const int type = a.type;
  const uint32_t N = a.N;
  const double* Q = a.Q + ((size_t)k * a.n_outer + p) * N;
  const Real* X = (const Real*)a.X;
  const Real* V = (const Real*)a.V;
  uint32_t ties = 0;
  double pi = 0.0, best = I.h0;  // date 0: Z_0 - pi_0
  for (uint32_t n = 0; n < N; ++n) {
    const uint32_t date = n + 1;
    const Real* t = tab + (size_t)date * kOosConsts;
    if (!CHK_OK(a.chk, t, sizeof(Real) * kOosConsts) ||
        !CHK_OK(a.chk, &scr[date], sizeof(ScreenConsts)) ||
        !CHK_OK(a.chk, &Q[n], sizeof(double) * (date < N ? 2 : 1)))
      break;
    const Real E = Fm<Real>::exp_(CHK_LD(a.chk, &X[(size_t)date * a.n_outer + p]), tabs);
    const Real S = t[7] * E;
    double Z, L;
    if (date < N) {
      Z = date_cash<Real>(t, type, K, S);
      double zx;
      const Real vs = stored_variance<Real>(SCHEME, CHK_LD(a.chk, &V[(size_t)date * a.n_outer + p]));
      L = rule_exercises<Real, BASIS>(t, scr[date], type, K, invK, invTh, E, vs, &zx, &ties)
              ? zx : Q[date];
    } else {
      Z = maturity_cash<Real>(t, type, K, S);
      L = Z;
    }
    pi += L - Q[n];
    best = fmax(best, Z - pi);
  }
  CHK_ST(a.chk, &a.dmax[(size_t)k * a.n_outer + p], best);
  CHK_ST(a.chk, &a.piN[(size_t)k * a.n_outer + p], pi);
  CHK_ST(a.chk, &a.max_ties[(size_t)k * a.n_outer + p], ties);
}

// Per strike (a CTA each): sums over outer paths in a fixed order, the
// bound, its standard error and the martingale's mean at maturity.
__global__ void dual_sum_kernel(DualArgs a) {
  const uint32_t k = blockIdx.x;
  __shared__ double s[5][kDualBlock];
  double d = 0.0, d2 = 0.0, q = 0.0, q2 = 0.0, tt = 0.0;
  for (uint32_t p = threadIdx.x; p < a.n_outer; p += kDualBlock) {
    const double x = CHK_LD(a.chk, &a.dmax[(size_t)k * a.n_outer + p]);
    const double y = CHK_LD(a.chk, &a.piN[(size_t)k * a.n_outer + p]);
    d += x; d2 += x * x; q += y; q2 += y * y;
    tt += (double)CHK_LD(a.chk, &a.max_ties[(size_t)k * a.n_outer + p]);
  }
  if (k == 0) {  // the inner rules' near ties, counted once
    const uint32_t cells = a.n_outer * a.N;
    for (uint32_t c = threadIdx.x; c < cells; c += kDualBlock)
      tt += (double)CHK_LD(a.chk, &a.inner_ties[c]);
  }
  s[0][threadIdx.x] = d; s[1][threadIdx.x] = d2; s[2][threadIdx.x] = q;
  s[3][threadIdx.x] = q2; s[4][threadIdx.x] = tt;
  __syncthreads();
  if (threadIdx.x < 5) {
    double v = 0.0;
    for (int i = 0; i < kDualBlock; ++i) v += s[threadIdx.x][i];
    s[threadIdx.x][0] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double n = (double)a.n_outer;
    const double mean = s[0][0] / n, mq = s[2][0] / n;
    const double var = a.n_outer > 1 ? (s[1][0] - n * mean * mean) / (n - 1.0) : 0.0;
    const double vq = a.n_outer > 1 ? (s[3][0] - n * mq * mq) / (n - 1.0) : 0.0;
    double* o = a.out + (size_t)k * kDualOut;
    if (!CHK_OK(a.chk, o, sizeof(double) * 5)) return;
    o[0] = mean;
    o[1] = var > 0.0 ? sqrt(var / n) : 0.0;
    o[2] = mq;
    o[3] = vq > 0.0 ? sqrt(vq / n) : 0.0;
    o[4] = s[4][0];
  }
}

template <typename Real, int SCHEME, int BASIS>
static cudaError_t launch_dual_t(const DualArgs& a, cudaStream_t s) {
  dual_outer_kernel<Real, SCHEME><<<(a.n_outer + kDualBlock - 1) / kDualBlock, kDualBlock, 0, s>>>(a);
  dual_inner_kernel<Real, SCHEME, BASIS><<<a.n_outer * a.N, kDualBlock, 0, s>>>(a);
  dual_max_kernel<Real, SCHEME, BASIS>
      <<<dim3((a.n_outer + kDualBlock - 1) / kDualBlock, a.n_strikes), kDualBlock, 0, s>>>(a);
  dual_sum_kernel<<<a.n_strikes, kDualBlock, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename Real>
static cudaError_t launch_dual_p(const DualArgs& a, int scheme, int basis, cudaStream_t s) {
  if (scheme == kSchemeQE)
    return basis == kBasisSV2 ? launch_dual_t<Real, kSchemeQE, kBasisSV2>(a, s)
                              : launch_dual_t<Real, kSchemeQE, kBasisS2>(a, s);
  return basis == kBasisSV2 ? launch_dual_t<Real, kSchemeFT, kBasisSV2>(a, s)
                            : launch_dual_t<Real, kSchemeFT, kBasisS2>(a, s);
}

cudaError_t launch_dual(const DualArgs& a, int precision, int scheme, int basis,
                        cudaStream_t s) {
  if (a.n_outer == 0 || a.N == 0 || a.n_strikes == 0 || a.n_strikes > kMaxDualStrikes ||
      a.n_inner == 0 || (uint64_t)a.n_outer * a.N + 1 > 0x7fffffffull)
    return cudaErrorInvalidValue;
  if (precision == kPrecFP64) return launch_dual_p<double>(a, scheme, basis, s);
  if (precision == kPrecDF) return launch_dual_p<df>(a, scheme, basis, s);
  return launch_dual_p<float>(a, scheme, basis, s);
}

}  // namespace lsmc
