// oos.cu -- out-of-sample Longstaff-Schwartz pricing pass.
//
// The coefficients of every date, fitted by the backward induction on the
// regression paths (cash flows discounted to t_0), are applied as a fixed
// exercise policy to an independent set of pricing paths (the same
// simulation on another stream, now in the instance's rows).  A pricing path
// stops at the first date n = 1..N-1 at which it is in the money and its
// discounted payoff beats the fitted continuation value -- the backward
// pass's own test, with the same operations -- else at maturity.  The mean
// of the stopped, discounted payoffs is a low-biased estimator of the
// American price (Longstaff and Schwartz, cited in Sec. 1).
//
// Work decomposition.  A CTA owns kOosTile paths of one instance; each
// thread owns kOosPpt of them and walks the dates forward.  At each date a
// warp compacts its in-the-money paths that have not stopped yet into a
// dense list in shared memory and runs the exercise test on the list, so the
// test's arithmetic is spent on candidates only, not on lanes whose paths
// are out of the money or already stopped.
#include <type_traits>

#include "checked.cuh"
#include "dfloat.cuh"
#include "exercise.cuh"
#include "kernels.h"
#include "plan.h"
#include "store16.cuh"

namespace lsmc {

namespace {

constexpr int kOosBlock = 128;                  // threads per CTA
constexpr int kOosPpt = kOosTile / kOosBlock;   // paths per thread
static_assert(kOosPpt * kOosBlock == kOosTile, "tile = block x paths per thread");
static_assert(kOosPpt <= 32, "the candidate mask is one word");

// solved flag of a date as written by the table kernel (exactly 0 or 1)
__device__ __forceinline__ bool flag_set(double f) { return __double_as_longlong(f) != 0; }
__device__ __forceinline__ bool flag_set(float f) { return __float_as_int(f) != 0; }
__device__ __forceinline__ bool flag_set(df f) { return __float_as_int(f.hi) != 0; }

// a stopped path's cash flow is non-negative; the initial marker is -1
// (sign tests on the integer pipe)
__device__ __forceinline__ bool stopped_value(double z) { return __double_as_longlong(z) >= 0; }
__device__ __forceinline__ bool stopped_value(float z) { return __float_as_int(z) >= 0; }
__device__ __forceinline__ bool stopped_value(df z) { return __float_as_int(z.hi) >= 0; }


// Shared memory of one warp: the compacted candidates of the current date
// (S, v and origin = slot * 32 + lane) and, by origin, the discounted cash
// flow of every path that has stopped (a negative value: not stopped; an
// exercised cash flow is positive).
template <typename Real, int BASIS>
struct OosWarpBufs {
  Real s[kOosPpt * 32];
  Real v[BASIS == kBasisSV2 ? kOosPpt * 32 : 1];
  Real z[kOosPpt][32];
  unsigned short o[kOosPpt * 32];
  unsigned short ex[kOosPpt * 32];  // items the float screen did not settle
};

}  // namespace

// The per-date constants of the pricing pass in the working precision,
// converted once per instance and date instead of once per path and date:
// coefficients, solved flag, S multiplier of the rows, discount factor
// exp(-r t_n) as a pair (hi, lo).  Dates without a regression (t_0, t_N, a
// European contract, a singular solve) get the flag 0.
template <typename Real>
__global__ void oos_table_kernel(const BwdInstance* __restrict__ inst CHK_PARAM) {
  if (!CHK_OK(chk, &inst[blockIdx.x], sizeof(BwdInstance))) return;
  const BwdInstance& I = inst[blockIdx.x];
  Real* tab = (Real*)I.oos_tab;
  const double* stab = I.scale_tab;
  const double* dtab = I.scale_tab + I.N + 1;
  for (uint32_t n = threadIdx.x; n <= I.N; n += blockDim.x) {
    Real* t = tab + (size_t)n * kOosConsts;
    const bool regress = n >= 1 && n < I.N && I.style == kAmerican;
    const double* bz = I.beta_z + (size_t)n * 8;
    if (!CHK_OK(chk, t, sizeof(Real) * kOosConsts) ||
        (regress && !CHK_OK(chk, bz, sizeof(double) * 7)) ||
        !CHK_OK(chk, &stab[n], sizeof(double)) || !CHK_OK(chk, &dtab[n], sizeof(double)) ||
        !CHK_OK(chk, &((ScreenConsts*)I.oos_screen)[n], sizeof(ScreenConsts)))
      continue;
    for (int i = 0; i < 6; ++i) t[i] = (Real)(regress ? bz[i] : 0.0);
    t[6] = (Real)(regress && bz[6] != 0.0 ? 1.0 : 0.0);
    t[7] = (Real)stab[n];
    const double d = dtab[n];
    t[8] = (Real)d;
    t[9] = (Real)(d - (double)(Real)d);
    t[10] = (Real)(std::is_same<Real, double>::value ? itm_threshold(I.type, stab[n], I.K) : 0.0);
    t[11] = (Real)0;
    // the float screen of the test (row value e, S = s e)
    ScreenConsts& q = ((ScreenConsts*)I.oos_screen)[n];
    float B = 0.0f;
    for (int i = 0; i < 6; ++i) {
      q.b[i] = (float)(double)t[i];
      B += fabsf(q.b[i]);
    }
    q.B = B;
    q.s = (float)(double)t[7];
    q.K = (float)I.K;
    q.invK = (float)I.invK;
    q.invTh = (float)I.inv_theta;
    q.d = (float)(double)t[8];
  }
}

template <typename Real, int BASIS, int FMT>
__global__ void __launch_bounds__(kOosBlock)
oos_kernel(const BwdInstance* __restrict__ inst CHK_PARAM) {
  using RR = RowRead<Real, FMT>;  // the E/V rows' elements and their widening
  using St = typename RR::raw;
  constexpr int PPT = kOosPpt;
  // the compacted list holds the row values e: double finds its candidates
  // without the product s1 e (threshold), and the float screen of the test
  // reads e; S = s1 e is formed on the list where the test needs it
  constexpr bool kScreen = !std::is_same<Real, float>::value;
  // consecutive CTAs take the same path tile of consecutive instances, so
  // the instances of one path group read the tile's rows while they are in L2
  if (!CHK_OK(chk, &inst[blockIdx.x], sizeof(BwdInstance))) return;  // the whole block
  const BwdInstance& I = inst[blockIdx.x];
  const uint32_t P = I.P, N = I.N;
  const uint32_t base = blockIdx.y * kOosTile;
  if (base >= P) return;  // the whole block
  __shared__ OosWarpBufs<Real, BASIS> s_wb[kOosBlock / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  OosWarpBufs<Real, BASIS>& wb = s_wb[warp];
  const unsigned lane_lt = (1u << lane) - 1u;
  const St* E = (const St*)I.E;
  const St* V = (const St*)I.V;
  const size_t ld = I.ld;
  const Real* tab = (const Real*)I.oos_tab;
  const int type = I.type;
  const Real K = (Real)I.K, invK = (Real)I.invK, invTh = (Real)I.inv_theta;
#pragma unroll
  for (int k = 0; k < PPT; ++k) wb.z[k][lane] = (Real)-1;
  __syncwarp();
  uint32_t valid = 0;    // bit k: slot k holds a path of the instance
#pragma unroll
  for (int k = 0; k < PPT; ++k)
    if (base + k * kOosBlock + tid < P) valid |= 1u << k;
  uint32_t stopped = 0;  // bit k: the path of slot k has exercised
  uint32_t ties = 0;
  if (I.style == kAmerican) {
    for (uint32_t n = 1; n < N; ++n) {
      // the warp leaves the date loop once none of its paths is live
      if (__all_sync(0xffffffffu, (valid & ~stopped) == 0u)) break;
      const Real* t = tab + (size_t)n * kOosConsts;
      if (!CHK_OK(chk, t, sizeof(Real) * kOosConsts)) continue;  // (uniform)
      if (!flag_set(t[6])) continue;  // no regression at n: no exercise (uniform)
      const Real s1 = t[7];
      const St* En = E + (size_t)(n - 1) * ld + base + tid;
      const St* Vn = BASIS == kBasisSV2 ? V + (size_t)(n - 1) * ld + base + tid : nullptr;
      // all loads of the date first, then the in-the-money tests
      St er[PPT], vr[PPT];
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        er[k] = vr[k] = (St)0;
        if (((valid & ~stopped) >> k) & 1u) {
          er[k] = CHK_LD(chk, &En[k * kOosBlock]);
          if (BASIS == kBasisSV2) vr[k] = CHK_LD(chk, &Vn[k * kOosBlock]);
        }
      }
      Real e[PPT], v[PPT];
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        e[k] = RR::widen(er[k]);
        v[k] = RR::widen(vr[k]);
      }
      uint32_t cand = 0;
      int cnt = 0;
      // double: the in-the-money test on the stored value's bits against the
      // date's threshold, so only candidates pay for the product s1 e
      const long long thr = threshold_bits(t[10]);
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        const bool itm = (((valid & ~stopped) >> k) & 1u) && itm_test(type, K, s1, e[k], thr);
        const unsigned m = __ballot_sync(0xffffffffu, itm);
        if (itm) {
          const int pos = cnt + __popc(m & lane_lt);
          wb.s[pos] = e[k];
          if (BASIS == kBasisSV2) wb.v[pos] = v[k];
          wb.o[pos] = (unsigned short)(k * 32 + lane);
          cand |= 1u << k;
        }
        cnt += __popc(m);
      }
      __syncwarp();
      if (cnt > 0) {
        Real b[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) b[i] = t[i];
        const Real d1 = t[8], d1lo = t[9];
        // the float screen of every item; those it does not settle as
        // continuing are compacted again for the working-precision work
        const ScreenConsts q = CHK_LD(chk, &((const ScreenConsts*)I.oos_screen)[n]);
        int cnt2 = 0;
        for (int j0 = 0; j0 < cnt; j0 += 32) {
          const int j = j0 + lane;
          int pre = 0;
          if (j < cnt) {
            pre = 2;
            if constexpr (kScreen)
              pre = exercise_screen<BASIS>(q, type, approx_float(wb.s[j]),
                                           BASIS == kBasisSV2 ? approx_float(wb.v[j]) : 0.0f);
          }
          const unsigned m = __ballot_sync(0xffffffffu, pre != 0);
          if (pre != 0) wb.ex[cnt2 + __popc(m & lane_lt)] = (unsigned short)(j | (pre << 12));
          cnt2 += __popc(m);
        }
        __syncwarp();
        for (int jj = lane; jj < cnt2; jj += 32) {
          const int code = wb.ex[jj], j = code & 0xfff, pre = code >> 12;
          const Real S = s1 * wb.s[j];
          const Real h = intrinsic<Real>(type, K, S);
          const Real hd = qmul(h, d1);
          bool exercise = pre == 1;
          if (pre == 2) {
            const Real x = qfma(S, invK, (Real)-1);
            Real c = qfma(qfma(b[2], x, b[1]), x, b[0]);
            if (BASIS == kBasisSV2) {
              const Real w = qfma(wb.v[j], invTh, (Real)-1);
              c = qfma(qfma(b[5], w, qfma(b[4], x, b[3])), w, c);
            }
            bool tie;
            decide<Real>(hd, c, exercise, tie);
            if (tie) ++ties;
          }
          if (exercise) {
            Real hz;
            if constexpr (std::is_same<Real, df>::value) hz = quick_two_sum(hd.hi, hd.lo);
            else hz = fma(h, d1, h * d1lo);
            const int o = wb.o[j];
            wb.z[o >> 5][o & 31] = hz;
          }
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < PPT; ++k)
          if (((cand >> k) & 1u) && stopped_value(wb.z[k][lane])) stopped |= 1u << k;
      }
      __syncwarp();
    }
  }
  const Real* tN = tab + (size_t)N * kOosConsts;
  const Real sN = CHK_LD(chk, &tN[7]), dNhi = CHK_LD(chk, &tN[8]), dNlo = CHK_LD(chk, &tN[9]);
  const St* EN = E + (size_t)(N - 1) * ld + base + tid;
  double sz = 0.0, sz2 = 0.0, euro = 0.0;
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    if (!((valid >> k) & 1u)) break;
    const Real SN = sN * RR::widen(CHK_LD(chk, &EN[k * kOosBlock]));
    const Real hN = payoff<Real>(type, K, SN);
    const double zN = (double)fma(hN, dNhi, hN * dNlo);
    const double z = ((stopped >> k) & 1u) ? (double)wb.z[k][lane] : zN;
    sz += z;
    sz2 += z * z;
    euro += zN;
  }
  // fixed-order block sums
  __shared__ double s_part[kOosBlock / 32][4];
  sz = warp_sum(sz);
  sz2 = warp_sum(sz2);
  euro = warp_sum(euro);
  ties = __reduce_add_sync(0xffffffffu, ties);
  if (lane == 0) {
    s_part[warp][0] = sz;
    s_part[warp][1] = sz2;
    s_part[warp][2] = euro;
    s_part[warp][3] = (double)ties;
  }
  __syncthreads();
  if (tid < 4) {
    double acc = 0.0;
    for (int w = 0; w < kOosBlock / 32; ++w) acc += s_part[w][tid];
    CHK_ST(chk, &I.oos_sum[(size_t)blockIdx.y * 4 + tid], acc);
  }
}

// The out-of-sample estimator of every instance: the tile sums added in tile
// order, the result written as the pricing result.
__global__ void oos_finish_kernel(const BwdInstance* __restrict__ inst, uint32_t n_inst,
                                  const BwdState* __restrict__ state,
                                  BwdResult* __restrict__ results CHK_PARAM) {
  const uint32_t i = blockIdx.x;
  if (i >= n_inst || threadIdx.x != 0) return;
  if (!CHK_OK(chk, &inst[i], sizeof(BwdInstance)) || !CHK_OK(chk, &state[i], sizeof(BwdState)))
    return;
  const BwdInstance& I = inst[i];
  const uint32_t tiles = (I.P + kOosTile - 1) / kOosTile;
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (uint32_t t = 0; t < tiles; ++t)
    for (int k = 0; k < 4; ++k) s[k] += CHK_LD(chk, &I.oos_sum[(size_t)t * 4 + k]);
  const double Pd = (double)I.P;
  const double mean = s[0] / Pd;
  const double var = I.P > 1 ? (s[1] - Pd * mean * mean) / (Pd - 1.0) : 0.0;
  BwdResult res;
  res.cont = mean;
  res.se = var > 0.0 ? sqrt(var / Pd) : 0.0;
  res.euro = s[2] / Pd;
  res.price = I.style == kEuropean ? mean : fmax(I.h0, mean);
  res.itm = state[i].itm;
  res.ties = state[i].ties + s[3];
  res.singular = state[i].singular;
  res.done = 1;
  CHK_ST(chk, &results[I.out_index], res);
}

template <typename Real, int FMT>
static void launch_oos_f(const BwdInstance* inst, dim3 grid, bool sv2, cudaStream_t s CHK_PARAM) {
  if (sv2) oos_kernel<Real, kBasisSV2, FMT><<<grid, kOosBlock, 0, s>>>(inst CHK_ARG(chk));
  else oos_kernel<Real, kBasisS2, FMT><<<grid, kOosBlock, 0, s>>>(inst CHK_ARG(chk));
}

template <typename Real>
static void launch_oos_t(const BwdInstance* inst, uint32_t n_inst, dim3 grid, bool sv2, int fmt,
                         cudaStream_t s CHK_PARAM) {
  oos_table_kernel<Real><<<n_inst, 128, 0, s>>>(inst CHK_ARG(chk));
  if (fmt == kStoreF16) launch_oos_f<Real, kStoreF16>(inst, grid, sv2, s CHK_ARG(chk));
  else if (fmt == kStoreBF16) launch_oos_f<Real, kStoreBF16>(inst, grid, sv2, s CHK_ARG(chk));
  else launch_oos_f<Real, kStoreNative>(inst, grid, sv2, s CHK_ARG(chk));
}

cudaError_t launch_oos(const BwdInstance* inst, uint32_t n_inst, uint32_t max_paths,
                       const BwdState* state, BwdResult* results, int precision, int basis,
                       int fmt, cudaStream_t s CHK_PARAM) {
  if (n_inst == 0 || max_paths == 0) return cudaSuccess;
  if (fmt < kStoreNative || fmt > kStoreBF16) return cudaErrorInvalidValue;
  const uint32_t tiles = (max_paths + kOosTile - 1) / kOosTile;
  if (tiles > 65535u || n_inst > 0x7fffffffu) return cudaErrorInvalidValue;
  const dim3 grid(n_inst, tiles);
  const bool sv2 = basis == kBasisSV2;
  if (precision == kPrecFP64) launch_oos_t<double>(inst, n_inst, grid, sv2, fmt, s CHK_ARG(chk));
  else if (precision == kPrecDF) launch_oos_t<df>(inst, n_inst, grid, sv2, fmt, s CHK_ARG(chk));
  else launch_oos_t<float>(inst, n_inst, grid, sv2, fmt, s CHK_ARG(chk));
  oos_finish_kernel<<<n_inst, 32, 0, s>>>(inst, n_inst, state, results CHK_ARG(chk));
  return cudaGetLastError();
}

}  // namespace lsmc
