// forward.cu -- random inputs and Heston path generation (forward pass).
//
// One thread owns one path of one contract and runs the whole time loop in
// registers (the GPU form of the paper's loop interchange, Sec. 4.1: the
// serial dependency along time stays inside a thread, independent paths fill
// the machine).  Per step it draws Philox4x32-10 once, maps the words to the
// uniform grid and two normal quantiles, then advances every path group of
// the contract with those same inputs (common random numbers) and stores
// exp(x) and v for the step as one coalesced row per group (step-major,
// path-minor: the layout of Sec. 4.1, Fig. "datalayout").
#include <cstdio>

#include <type_traits>

#include "device_common.cuh"
#include "df_math.cuh"
#include "dfloat.cuh"
#include "kernels.h"
#include "plan.h"
#include "checked.cuh"
#include "heston_step.cuh"
#include "store16.cuh"

namespace lsmc {

// SEG: the launch covers dates (n0, n1] and may start from, or save, states
// (regenerate mode); without it, the whole horizon from the initial state
// into the full row store (the hot loop stays free of the segment logic).
template <typename Real, int SCHEME, bool SEG, int FMT>
// register budgets: 128 per thread for double, 64 for float (eight CTAs of
// 128 threads per SM), unconstrained for float pairs
__global__ void __launch_bounds__(kFwdBlock, std::is_same<Real, double>::value ? 4 : (std::is_same<Real, float>::value ? 8 : 1))
forward_kernel(FwdArgs a) {
  using St = typename StoreElem<Real, FMT>::type;  // element of the E/V rows
  __shared__ GroupConst<Real> gc[kMaxGroups];
  __shared__ FwdContract sc;
  if (threadIdx.x == 0) {
    // contract of this block: last contract whose block0 <= blockIdx.x
    uint32_t lo = 0, hi = a.n_contracts;
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) / 2;
      if (CHK_LD(a.chk, &a.contracts[mid].block0) <= blockIdx.x) lo = mid; else hi = mid;
    }
    if (CHK_OK(a.chk, &a.contracts[lo], sizeof(FwdContract))) sc = a.contracts[lo];
    else sc = FwdContract{};
  }
  __syncthreads();
  if (threadIdx.x < sc.n_groups && threadIdx.x < kMaxGroups &&
      CHK_OK(a.chk, &a.groups[sc.group0 + threadIdx.x], sizeof(FwdGroup)))
    make_group_const<Real>(a.groups[sc.group0 + threadIdx.x], gc[threadIdx.x]);
  // float pairs: exp and quantile tables in shared memory
  constexpr bool kPair = std::is_same<Real, df>::value;
  __shared__ __align__(16) unsigned char tab_raw[kPair ? sizeof(DfTables) : 16];
  DfTables* tabs = reinterpret_cast<DfTables*>(tab_raw);
  if constexpr (kPair) load_df_tables(tabs);
  __syncthreads();

  if (SEG && a.next_job && blockIdx.x == 0 && threadIdx.x == 0)
    CHK_ST(a.chk, a.next_job, a.next_job_value);
  const uint32_t p = (blockIdx.x - sc.block0) * kFwdBlock + threadIdx.x;
  if (p >= sc.P) return;
  const int ng = (int)sc.n_groups;
  const uint2 key = make_uint2((uint32_t)sc.seed, (uint32_t)(sc.seed >> 32));
  // dates (n0, n1] of this launch; the state at n0 is the initial one or a
  // saved one; E/V row of date d at index d - row0
  const uint32_t n0 = SEG ? a.n0 : 0u, n1 = SEG && a.n1 ? a.n1 : sc.N;
  const uint32_t row0 = SEG ? a.row0 : 1u;
  const bool store_rows = SEG ? a.store_rows != 0 : true;
  const size_t ck_index = SEG && a.ck_stride && n0 ? (size_t)(n0 / a.ck_stride) : 0;
  const bool first_row = SEG && store_rows && n0 >= row0;  // a segment: row of date n0 too
  auto save_at = [&](uint32_t d) {  // save the state after date d?
    return SEG && a.save_states && d % a.ck_stride == 0 && d < sc.N;
  };

  for (int g = 0; g < ng; ++g) {
    const FwdGroup& gg = a.groups[sc.group0 + g];
    if (gg.E_row0) CHK_ST(a.chk, &((St*)gg.E_row0)[p], narrow<St>(gc[g].out_scale));
    if (gg.V_row0) CHK_ST(a.chk, &((St*)gg.V_row0)[p], narrow<St>(gc[g].v0));
  }

  if constexpr (std::is_same<Real, float>::value && SCHEME == kSchemeQE) {
    // the single-precision QE stepper: state, scheme constants and row
    // pointers of every group in registers, the group loop unrolled so the
    // groups' independent chains interleave, one shared row offset
    float x[kMaxGroups], v[kMaxGroups], mA[kMaxGroups], mB[kMaxGroups], sA[kMaxGroups],
        sB[kMaxGroups], c0[kMaxGroups], K1[kMaxGroups], K2[kMaxGroups], K3[kMaxGroups],
        os[kMaxGroups];
    St* rowE[kMaxGroups];
    St* rowV[kMaxGroups];
#pragma unroll
    for (int g = 0; g < kMaxGroups; ++g) {
      const GroupConst<float>& c = gc[g < ng ? g : 0];
      x[g] = 0.0f;
      v[g] = c.v0;
      mA[g] = c.mA; mB[g] = c.mB; sA[g] = c.sA; sB[g] = c.sB;
      c0[g] = c.c0; K1[g] = c.K1; K2[g] = c.K2; K3[g] = c.K3;
      os[g] = c.out_scale;
      rowE[g] = (St*)c.E + p;
      rowV[g] = c.V ? (St*)c.V + p : nullptr;
    }
    const size_t ld = gc[0].ld;  // one row stride for the groups of a contract
    if (ck_index) {
#pragma unroll
      for (int g = 0; g < kMaxGroups; ++g)
        if (g < ng) {
          x[g] = CHK_LD(a.chk, &gc[g].CX[ck_index * ld + p]);
          v[g] = CHK_LD(a.chk, &gc[g].CV[ck_index * ld + p]);
        }
    }
    if (first_row) {
#pragma unroll
      for (int g = 0; g < kMaxGroups; ++g)
        if (g < ng) {
          CHK_ST(a.chk, &rowE[g][0], narrow<St>(os[g] * __expf(x[g])));
          if (rowV[g]) CHK_ST(a.chk, &rowV[g][0], narrow<St>(v[g]));
        }
    }
    // the time loop, once with every group present, storing v and with unit
    // row scale, under the launch's one key (the full bump set with the SV2
    // basis in a plan: no per-group or per-store tests, no scaling and no key
    // schedule in the loop), once for the general case
    auto time_loop = [&](auto all_groups) {
      constexpr bool kAll = decltype(all_groups)::value;
      size_t off = (size_t)(n0 + 1 - row0) * ld;
      for (uint32_t n = n0; n < n1; ++n, off += ld) {
        const uint4 ctr = make_uint4(p, n, sc.stream_id ^ a.stream_xor, 0u);
        const uint4 w = kAll ? philox4x32_10_rk(ctr, a.rk) : philox4x32_10(ctr, key);
        float u, omu, zV, zX;
        Draw<float>::make(w, u, omu, zV, zX, tabs);
#pragma unroll
        for (int g = 0; g < kMaxGroups; ++g) {
          if (kAll || g < ng) {
            float xg = x[g], vg = v[g];
            qe_core<float>(mA[g], mB[g], sA[g], sB[g], c0[g], K1[g], K2[g], K3[g], xg, vg, omu,
                           zV, zX, tabs);
            x[g] = xg;
            v[g] = vg;
            if (store_rows) {
              CHK_ST(a.chk, &rowE[g][off], narrow<St>(kAll ? __expf(xg) : os[g] * __expf(xg)));
              if (kAll || rowV[g]) CHK_ST(a.chk, &rowV[g][off], narrow<St>(vg));
            }
            if (save_at(n + 1)) {
              CHK_ST(a.chk, &gc[g].CX[(size_t)((n + 1) / a.ck_stride) * ld + p], xg);
              CHK_ST(a.chk, &gc[g].CV[(size_t)((n + 1) / a.ck_stride) * ld + p], vg);
            }
          }
        }
      }
    };
    bool all = ng == kMaxGroups;
#pragma unroll
    for (int g = 0; g < kMaxGroups; ++g) all = all && rowV[g] != nullptr && os[g] == 1.0f;
    all = all && a.uniform_key != 0;
    if (all) time_loop(std::true_type{});
    else time_loop(std::false_type{});
  } else if constexpr (!kPair) {
    // double (and the float Euler scheme): every group's state in registers,
    // the group loop unrolled so the groups' independent chains interleave
    Real x[kMaxGroups], v[kMaxGroups];
#pragma unroll
    for (int g = 0; g < kMaxGroups; ++g) {
      x[g] = (Real)0;
      v[g] = g < ng ? gc[g].v0 : (Real)0;
      if (ck_index && g < ng) {
        x[g] = CHK_LD(a.chk, &gc[g].CX[ck_index * gc[g].ld + p]);
        v[g] = CHK_LD(a.chk, &gc[g].CV[ck_index * gc[g].ld + p]);
      }
      if (first_row && g < ng) {
        const GroupConst<Real>& c = gc[g];
        CHK_ST(a.chk, &((St*)c.E)[p], narrow<St>(c.out_scale * Fm<Real>::exp_(x[g], tabs)));
        if (c.V)
          CHK_ST(a.chk, &((St*)c.V)[p],
                 narrow<St>((SCHEME == kSchemeFT && v[g] < (Real)0) ? (Real)0 : v[g]));
      }
    }
    for (uint32_t n = n0; n < n1; ++n) {
      const uint4 w = philox4x32_10(make_uint4(p, n, sc.stream_id ^ a.stream_xor, 0u), key);
      Real u, omu, zV, zX;
      Draw<Real>::make(w, u, omu, zV, zX, tabs);
#pragma unroll
      for (int g = 0; g < kMaxGroups; ++g) {
        if (g < ng) {
          const GroupConst<Real>& c = gc[g];
          if (SCHEME == kSchemeQE) {
            qe_step<Real>(c, x[g], v[g], omu, zV, zX, tabs);
          } else {
            ft_step<Real>(c, x[g], v[g], zV, zX);
          }
          if (store_rows) {
            const size_t off = (size_t)(n + 1 - row0) * c.ld + p;
            CHK_ST(a.chk, &((St*)c.E)[off], narrow<St>(c.out_scale * Fm<Real>::exp_(x[g], tabs)));
            if (c.V)
              CHK_ST(a.chk, &((St*)c.V)[off],
                     narrow<St>((SCHEME == kSchemeFT && v[g] < (Real)0) ? (Real)0 : v[g]));
          }
          if (save_at(n + 1)) {
            CHK_ST(a.chk, &c.CX[(size_t)((n + 1) / a.ck_stride) * c.ld + p], x[g]);
            CHK_ST(a.chk, &c.CV[(size_t)((n + 1) / a.ck_stride) * c.ld + p], v[g]);
          }
        }
      }
    }
  } else {
    // float pairs: a group step is several hundred instructions, so the
    // group loop is not unrolled (the code stays in the instruction cache)
    // and the per-group state lives in shared memory
    __shared__ Real xs[kMaxGroups][kFwdBlock], vs[kMaxGroups][kFwdBlock];
    const int t = threadIdx.x;
    for (int g = 0; g < ng; ++g) {
      const GroupConst<Real>& c = gc[g];
      xs[g][t] = ck_index ? CHK_LD(a.chk, &c.CX[ck_index * c.ld + p]) : (Real)0;
      vs[g][t] = ck_index ? CHK_LD(a.chk, &c.CV[ck_index * c.ld + p]) : c.v0;
      if (first_row) {
        CHK_ST(a.chk, &((St*)c.E)[p], narrow<St>(c.out_scale * Fm<Real>::exp_(xs[g][t], tabs)));
        if (c.V)
          CHK_ST(a.chk, &((St*)c.V)[p],
                 narrow<St>((SCHEME == kSchemeFT && vs[g][t] < (Real)0) ? (Real)0 : vs[g][t]));
      }
    }
    for (uint32_t n = n0; n < n1; ++n) {
      const uint4 w = philox4x32_10(make_uint4(p, n, sc.stream_id ^ a.stream_xor, 0u), key);
      Real u, omu, zV, zX;
      Draw<Real>::make(w, u, omu, zV, zX, tabs);
#pragma unroll 1
      for (int g = 0; g < ng; ++g) {
        const GroupConst<Real>& c = gc[g];
        Real xg = xs[g][t], vg = vs[g][t];
        if (SCHEME == kSchemeQE) {
          qe_step<Real>(c, xg, vg, omu, zV, zX, tabs);
        } else {
          ft_step<Real>(c, xg, vg, zV, zX);
        }
        xs[g][t] = xg;
        vs[g][t] = vg;
        if (store_rows) {
          const size_t off = (size_t)(n + 1 - row0) * c.ld + p;
          CHK_ST(a.chk, &((St*)c.E)[off], narrow<St>(c.out_scale * Fm<Real>::exp_(xg, tabs)));
          if (c.V)
            CHK_ST(a.chk, &((St*)c.V)[off],
                   narrow<St>((SCHEME == kSchemeFT && vg < (Real)0) ? (Real)0 : vg));
        }
        if (save_at(n + 1)) {
          CHK_ST(a.chk, &c.CX[(size_t)((n + 1) / a.ck_stride) * c.ld + p], xg);
          CHK_ST(a.chk, &c.CV[(size_t)((n + 1) / a.ck_stride) * c.ld + p], vg);
        }
      }
    }
  }
}

// ---- STAC-A2 multi-asset path reduction (Sec. 2.2.1, Sec. 4.1) ---------------
// M[n][p] = max over assets of S_a[n][p].  Like the paper's loop interchange,
// the assets are the outer loop of a thread (KA of them at a time, their
// state in registers and their steps interleaved), the dates the inner
// loop, and the running maximum lives in M itself (read, compared, written
// back by the one thread that owns the path).  Element (path, asset, date)
// draws from Philox counter (path, date, stream, asset); the common
// log-price shock of (path, date), used when the assets are correlated,
// from counter (path, date, stream, 0xFFFFFFFF).

template <typename Real>
__device__ __forceinline__ Real common_shock(uint4 w, const DfTables* t);
template <>
__device__ __forceinline__ double common_shock<double>(uint4 w, const DfTables*) {
  const double u = uniform52(w.z, w.w);
  return norm_quantile_f64(u, 1.0 - u);
}
template <>
__device__ __forceinline__ float common_shock<float>(uint4 w, const DfTables*) {
  const float u = uniform23(w.z);
  return norm_quantile_f32(u, 1.0f - u);
}
template <>
__device__ __forceinline__ df common_shock<df>(uint4 w, const DfTables* t) {
  return Draw<df>::quantile(w.z, w.w, t);
}

template <typename Real, int SCHEME, int KA>
__global__ void __launch_bounds__(kFwdBlock)
multi_max_kernel(MultiArgs a) {
  __shared__ GroupConst<Real> gc[kMaxAssets];
  constexpr bool kPair = std::is_same<Real, df>::value;
  __shared__ __align__(16) unsigned char tab_raw[kPair ? sizeof(DfTables) : 16];
  DfTables* tabs = reinterpret_cast<DfTables*>(tab_raw);
  if constexpr (kPair) load_df_tables(tabs);
  const double dt = a.T / (double)a.N;
  for (uint32_t i = threadIdx.x; i < a.n_assets; i += blockDim.x) {
    const MultiModel& m = a.assets[i];
    FwdGroup g{};
    g.v0 = m.v0; g.kappa = m.kappa; g.theta = m.theta; g.xi = m.xi; g.rho = m.rho;
    g.r = m.r; g.q = m.q; g.dt = dt; g.out_scale = m.S0;
    make_group_const<Real>(g, gc[i]);
  }
  __syncthreads();
  const uint32_t p = blockIdx.x * kFwdBlock + threadIdx.x;
  if (p >= a.P) return;
  const uint2 key = make_uint2((uint32_t)a.seed, (uint32_t)(a.seed >> 32));
  const bool corr = a.sqrt_rho > 0.0;
  const Real sr = (Real)a.sqrt_rho, s1r = (Real)a.sqrt_1m_rho;
  Real* M = (Real*)a.M;
  const size_t P = a.P;

  for (uint32_t a0 = 0; a0 < a.n_assets; a0 += KA) {
    Real x[KA], v[KA];
    Real m0 = (Real)0;
#pragma unroll
    for (int k = 0; k < KA; ++k) {
      const uint32_t ai = a0 + k < a.n_assets ? a0 + k : a0;
      x[k] = (Real)0;
      v[k] = gc[ai].v0;
      if (k == 0 || gc[ai].out_scale > m0) m0 = gc[ai].out_scale;
    }
    CHK_ST(a.chk, &M[p], a0 == 0 ? m0 : fmax(CHK_LD(a.chk, &M[p]), m0));
    for (uint32_t n = 0; n < a.N; ++n) {
      Real zc = (Real)0;
      if (corr)
        zc = common_shock<Real>(philox4x32_10(make_uint4(p, n, a.stream_id, 0xFFFFFFFFu), key),
                                tabs);
      Real mx = (Real)0;
#pragma unroll
      for (int k = 0; k < KA; ++k) {
        if (a0 + k < a.n_assets) {
          const GroupConst<Real>& c = gc[a0 + k];
          const uint4 w = philox4x32_10(make_uint4(p, n, a.stream_id, a0 + k), key);
          Real u, omu, zV, zX;
          Draw<Real>::make(w, u, omu, zV, zX, tabs);
          if (corr) zX = sr * zc + s1r * zX;
          if (SCHEME == kSchemeQE) {
            qe_step<Real>(c, x[k], v[k], omu, zV, zX, tabs);
          } else {
            ft_step<Real>(c, x[k], v[k], zV, zX);
          }
          const Real S = c.out_scale * Fm<Real>::exp_(x[k], tabs);
          mx = k == 0 ? S : fmax(mx, S);
        }
      }
      const size_t off = (size_t)(n + 1) * P + p;
      CHK_ST(a.chk, &M[off], a0 == 0 ? mx : fmax(CHK_LD(a.chk, &M[off]), mx));
    }
  }
}

template <typename Real>
static void launch_multi_t(const MultiArgs& a, int scheme, cudaStream_t s) {
  const unsigned blocks = (a.P + kFwdBlock - 1) / kFwdBlock;
  if (scheme == kSchemeQE)
    multi_max_kernel<Real, kSchemeQE, 4><<<blocks, kFwdBlock, 0, s>>>(a);
  else
    multi_max_kernel<Real, kSchemeFT, 4><<<blocks, kFwdBlock, 0, s>>>(a);
}

cudaError_t launch_multi_max(const MultiArgs& a, int precision, int scheme, cudaStream_t s) {
  if (a.P == 0 || a.N == 0 || a.n_assets == 0) return cudaSuccess;
  if (precision == kPrecFP64) launch_multi_t<double>(a, scheme, s);
  else if (precision == kPrecDF) launch_multi_t<df>(a, scheme, s);
  else launch_multi_t<float>(a, scheme, s);
  return cudaGetLastError();
}

// The exponential of the forward pass (the E rows are S0 exp(x)): exp_f64
// in double, exp_df on float pairs, __expf in single precision.
template <typename Real>
__global__ void exp_kernel(const Real* __restrict__ x, Real* __restrict__ y, size_t n) {
  constexpr bool kPair = std::is_same<Real, df>::value;
  __shared__ __align__(16) unsigned char tab_raw[kPair ? sizeof(DfTables) : 16];
  DfTables* tabs = reinterpret_cast<DfTables*>(tab_raw);
  if constexpr (kPair) {
    load_df_tables(tabs);
    __syncthreads();
  }
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = Fm<Real>::exp_(x[i], tabs);
}

// The normal quantile of the random inputs on n uniforms (1 - u computed;
// exact on the precision's uniform grid).
template <typename Real>
__global__ void quantile_kernel(const Real* __restrict__ u, Real* __restrict__ z, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Real ui = u[i];
  if constexpr (std::is_same<Real, double>::value) z[i] = norm_quantile_f64(ui, 1.0 - ui);
  else z[i] = norm_quantile_f32(ui, 1.0f - ui);
}

cudaError_t launch_quantile(const void* u, void* z, size_t n, int precision, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const size_t blocks = (n + kBlock - 1) / kBlock;
  if (blocks > 0x7fffffffu) return cudaErrorInvalidValue;
  if (precision == kPrecFP64)
    quantile_kernel<double><<<(unsigned)blocks, kBlock, 0, s>>>((const double*)u, (double*)z, n);
  else
    quantile_kernel<float><<<(unsigned)blocks, kBlock, 0, s>>>((const float*)u, (float*)z, n);
  return cudaGetLastError();
}

cudaError_t launch_exp(const void* x, void* y, size_t n, int precision, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const size_t blocks = (n + kBlock - 1) / kBlock;
  if (blocks > 0x7fffffffu) return cudaErrorInvalidValue;
  if (precision == kPrecFP64)
    exp_kernel<double><<<(unsigned)blocks, kBlock, 0, s>>>((const double*)x, (double*)y, n);
  else if (precision == kPrecDF)
    exp_kernel<df><<<(unsigned)blocks, kBlock, 0, s>>>((const df*)x, (df*)y, n);
  else
    exp_kernel<float><<<(unsigned)blocks, kBlock, 0, s>>>((const float*)x, (float*)y, n);
  return cudaGetLastError();
}

__global__ void philox_kernel(const uint4* __restrict__ ctr, uint2 key,
                              uint4* __restrict__ out, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = philox4x32_10(ctr[i], key);
}

template <typename Real>
__global__ void draws_kernel(uint2 key, uint32_t stream_id,
                             const uint32_t* __restrict__ path,
                             const uint32_t* __restrict__ step, size_t n,
                             Real* __restrict__ out) {
  constexpr bool kPair = std::is_same<Real, df>::value;
  __shared__ __align__(16) unsigned char tab_raw[kPair ? sizeof(DfTables) : 16];
  DfTables* tabs = reinterpret_cast<DfTables*>(tab_raw);
  if constexpr (kPair) {
    load_df_tables(tabs);
    __syncthreads();
  }
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 w = philox4x32_10(make_uint4(path[i], step[i], stream_id, 0u), key);
  Real uV, omu, zV, zX;
  Draw<Real>::make(w, uV, omu, zV, zX, tabs);
  out[3 * i] = uV;
  out[3 * i + 1] = zV;
  out[3 * i + 2] = zX;
}

template <typename Real, int FMT>
static void launch_forward_f(const FwdArgs& a, int scheme, cudaStream_t s) {
  const bool seg = a.n0 != 0 || a.n1 != 0 || a.row0 != 1 || !a.store_rows || a.save_states ||
                   a.next_job;
  if (scheme == kSchemeQE) {
    if (seg) forward_kernel<Real, kSchemeQE, true, FMT><<<a.n_blocks, kFwdBlock, 0, s>>>(a);
    else forward_kernel<Real, kSchemeQE, false, FMT><<<a.n_blocks, kFwdBlock, 0, s>>>(a);
  } else {
    if (seg) forward_kernel<Real, kSchemeFT, true, FMT><<<a.n_blocks, kFwdBlock, 0, s>>>(a);
    else forward_kernel<Real, kSchemeFT, false, FMT><<<a.n_blocks, kFwdBlock, 0, s>>>(a);
  }
}

template <typename Real>
static void launch_forward_t(const FwdArgs& a, int scheme, cudaStream_t s) {
  if (a.store_fmt == kStoreF16) launch_forward_f<Real, kStoreF16>(a, scheme, s);
  else if (a.store_fmt == kStoreBF16) launch_forward_f<Real, kStoreBF16>(a, scheme, s);
  else launch_forward_f<Real, kStoreNative>(a, scheme, s);
}

cudaError_t launch_forward(const FwdArgs& a, int precision, int scheme, cudaStream_t s) {
  if (a.n_blocks == 0) return cudaSuccess;
  if (a.store_fmt < kStoreNative || a.store_fmt > kStoreBF16) return cudaErrorInvalidValue;
  if (precision == kPrecFP64) launch_forward_t<double>(a, scheme, s);
  else if (precision == kPrecDF) launch_forward_t<df>(a, scheme, s);
  else launch_forward_t<float>(a, scheme, s);
  return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1,
                          uint32_t* out, size_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const size_t blocks = (n + kBlock - 1) / kBlock;
  philox_kernel<<<(unsigned)blocks, kBlock, 0, s>>>(
      (const uint4*)ctr, make_uint2(k0, k1), (uint4*)out, n);
  return cudaGetLastError();
}

cudaError_t launch_draws(uint64_t seed, uint32_t stream_id, const uint32_t* path,
                         const uint32_t* step, size_t n, int precision, void* out,
                         cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const size_t blocks = (n + kBlock - 1) / kBlock;
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  if (precision == kPrecFP64)
    draws_kernel<double><<<(unsigned)blocks, kBlock, 0, s>>>(key, stream_id, path, step, n, (double*)out);
  else if (precision == kPrecDF)
    draws_kernel<df><<<(unsigned)blocks, kBlock, 0, s>>>(key, stream_id, path, step, n, (df*)out);
  else
    draws_kernel<float><<<(unsigned)blocks, kBlock, 0, s>>>(key, stream_id, path, step, n, (float*)out);
  return cudaGetLastError();
}

}  // namespace lsmc
