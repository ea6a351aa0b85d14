// capi.cpp -- the extern "C" boundary: contexts, plans, synchronous pricing,
// stage entry points and the continuous-batching request loop.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/lsmc.h"
#include "kernels.h"
#include "plan.h"
#include "planner.h"

using namespace lsmc;

static_assert(sizeof(DevResult) == sizeof(lsmc_result), "result layout");
static_assert(offsetof(DevResult, status) == offsetof(lsmc_result, status), "result layout");
static_assert(offsetof(DevResult, n_near_ties) == offsetof(lsmc_result, n_near_ties), "result layout");
static_assert(offsetof(BwdResult, ties) == 4 * sizeof(double), "stage output layout");
static_assert(kScCount == LSMC_SC_COUNT && kScBase == LSMC_SC_BASE && kScVUp == LSMC_SC_V0_UP &&
                  kScTUp == LSMC_SC_T_UP, "scenario kinds");

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// device allocations made by the library in this process (cudaMalloc,
// cudaMallocAsync and the callbacks of lsmc_set_allocator; sub-allocations
// from a workspace are not counted): lsmc_device_allocations
std::atomic<uint64_t> g_device_allocs{0};
void count_device_alloc() { g_device_allocs.fetch_add(1, std::memory_order_relaxed); }

struct Ticket;

// A serving slot: one stream and, while busy, one plan pricing a batch of
// admitted tickets.  A request whose revaluations have all finished is
// handed over ahead of the rest of its batch: the backward pass writes its
// results to the slot's host-mapped array and raises its flag.
struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  std::vector<Ticket*> batch;  // null once a ticket finished ahead of its batch
  std::vector<uint32_t> nk;    // strikes of each batch entry
  lsmc_plan* plan = nullptr;
  DevResult* map_out = nullptr;  // host-mapped: results of the batch's strikes
  uint32_t* map_flag = nullptr;  // host-mapped: per request, set once its results are in
  size_t cap_out = 0, cap_req = 0;
};

}  // namespace

struct lsmc_ctx {
  int device = 0;
  int precision = LSMC_FP64, scheme = LSMC_SCHEME_QE;
  cudaStream_t own_stream = nullptr, stream = nullptr;
  Arena arena;
  bool user_workspace = false;
  void* own_arena_mem = nullptr;
  size_t hbm_budget = 0;
  uint32_t max_inflight = 8, queue_capacity = 4096;
  uint32_t max_batch = 64;    // requests admitted together (lsmc_config.max_batch)
  double serve_share = 0.0;   // share of the resident backward CTAs a batch takes (0: 1/slots)
  int num_sms = 0;
  std::map<int, int> occ;     // resident backward CTAs per SM by kernel variant
  std::mutex occ_mu;          // guards occ (plans are built on several threads)
  // device memory callbacks (lsmc_set_allocator); null: cudaMalloc / cudaFree
  void* (*dev_alloc)(size_t, void*) = nullptr;
  void (*dev_free)(void*, void*) = nullptr;
  void* alloc_user = nullptr;
  uint32_t sub_override = 0;  // backward sub-tiles per job | LSMC_SUB_ITM_HALF (0: chosen per plan)
  uint32_t ppt_override = 0;  // backward paths per lane (0: chosen per plan)
  double wait_limit_s = 20.0; // bound of every device-side wait (lsmc_set_wait_limit)
  // autotuned backward shape (ppt << 16 | sub-tiles per job | LSMC_SUB_ITM_HALF), keyed by
  // (precision, basis, log2 of the first round's sub-tile count)
  std::map<uint64_t, uint32_t> tuned;
  // serving
  std::mutex mu;
  std::condition_variable cv, done_cv;
  std::thread sched;
  bool stop = false, sched_started = false;
  std::deque<Ticket*> pending;
  std::map<uint64_t, Ticket*> tickets;
  uint64_t next_ticket = 1;
  std::vector<Slot> slots;
  double t0 = 0;
  // submit / admit / done times of released tickets (bounded history)
  std::map<uint64_t, std::array<double, 3>> history;
};

struct lsmc_plan {
  lsmc_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  PlanLayout L;
  char* dev = nullptr;
  int alloc_kind = 0;  // 0 cudaMalloc, 1 arena, 2 cudaMallocAsync, 3 the context's allocator
  bool run_forward = true, run_backward = true, run_greeks = true;
  FwdArgs fa{};
  BwdArgs ba{};
  BwdInstance* d_inst = nullptr;
  GreekOut* d_greeks = nullptr;
  BwdResult* d_results = nullptr;
  DevResult* d_out = nullptr;
  void* d_state = nullptr;
  size_t state_bytes = 0;
  Control* d_ctl = nullptr;
  int bwd_grid = 1;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<DevResult> h_out;
  std::vector<BwdResult> h_res;
  uint64_t itm = 0;
  // per-kernel timing: one set of 5 events per launch since the last read
  bool timing = false;
  std::vector<std::array<cudaEvent_t, 5>> ev;
  size_t ev_used = 0;
#ifdef LSMC_CHECKED
  CheckRanges chk{};  // the byte ranges the plan's launches may touch
#endif
};

namespace {

struct Ticket {
  uint64_t id = 0;
  lsmc_request req{};
  std::vector<double> strikes;
  int status = LSMC_PENDING;
  std::vector<lsmc_result> results;
  double t_submit = 0, t_admit = 0, t_done = 0;
  size_t footprint = 0;
  int slot = -1;
  // backward shape of this request priced alone (a batch keeps it, so a
  // result does not depend on the batch it ran in)
  uint32_t ppt = 0, sub = 1;
  int precision = 0, scheme = 0, basis = 0;
};

#ifdef LSMC_CHECKED
// one more byte range a checked launch may touch
void add_range(CheckRanges& c, const void* q, size_t bytes) {
  if (!q || !bytes || c.n >= (uint32_t)kMaxRanges) return;
  c.lo[c.n] = (unsigned long long)q;
  c.hi[c.n] = c.lo[c.n] + bytes;
  ++c.n;
}
#endif

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return LSMC_OK;
  if (e == cudaErrorMemoryAllocation) return LSMC_ENOMEM;
  return LSMC_ECUDA;
}

#define LSMC_CUDA(call)                          \
  do {                                           \
    cudaError_t e__ = (call);                    \
    if (e__ != cudaSuccess) return cuda_status(e__); \
  } while (0)

int resolve(const lsmc_ctx*, int32_t v, int dflt) { return v < 0 ? dflt : v; }

int occupancy(lsmc_ctx* ctx, int precision, int basis, int ppt, int fmt) {
  if (ctx) {
    std::lock_guard<std::mutex> g(ctx->occ_mu);
    int& o = ctx->occ[((precision * 4 + basis) * 16 + ppt) * 4 + fmt];
    if (o == 0) o = std::max(1, backward_occupancy(precision, basis, ppt, fmt));
    return o;
  }
  return std::max(1, backward_occupancy(precision, basis, ppt, fmt));
}

int sm_count(lsmc_ctx* ctx) {
  if (ctx && ctx->num_sms) return ctx->num_sms;
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  if (ctx) ctx->num_sms = n;
  return n > 0 ? n : 1;
}

// Device layout of a plan: tables | state + control | results | out |
// scale tables | partials | Y | paths.
int plan_bind_and_upload(lsmc_plan* p, void* ext_S, void* ext_V, double* beta_hist) {
  PlanLayout& L = p->L;
  const int prec = L.opt.precision;
  const size_t real = value_bytes(prec);
  char* base = p->dev;
  size_t off = 0;
  auto take = [&](size_t bytes) { char* q = base + off; off += align256(bytes); return q; };
  // tables (host blob mirrors this layout)
  std::vector<char> blob(L.bytes_tables, 0);
  size_t boff = 0;
  auto put = [&](const void* src, size_t bytes) -> char* {
    char* dst = base + boff;
    if (bytes) std::memcpy(blob.data() + boff, src, bytes);
    boff += align256(bytes);
    return dst;
  };
  char* paths = base + L.bytes_tables + L.bytes_state + L.bytes_results + L.bytes_out +
                L.bytes_scale + L.bytes_partial + L.bytes_y;
  char* yreg = paths - L.bytes_y;
  char* preg = yreg - L.bytes_partial;
  char* sreg = preg - L.bytes_scale;
  // bind group rows
  for (size_t g = 0; g < L.groups.size(); ++g) {
    FwdGroup& G = L.groups[g];
    if (ext_S) {
      G.E = (char*)ext_S + (size_t)G.ld * real;  // row 1 (ld == P here)
      G.E_row0 = ext_S;
      G.V = ext_V ? (char*)ext_V + (size_t)G.ld * real : nullptr;
      G.V_row0 = ext_V;
    } else {
      G.E = paths + L.group_E_off[g];
      G.V = L.group_V_off[g] == SIZE_MAX ? nullptr : paths + L.group_V_off[g];
      G.E_row0 = G.V_row0 = nullptr;
      G.CX = L.group_CX_off[g] == SIZE_MAX ? nullptr : paths + L.group_CX_off[g];
      G.CV = L.group_CV_off[g] == SIZE_MAX ? nullptr : paths + L.group_CV_off[g];
    }
  }
  for (size_t i = 0; i < L.inst.size(); ++i) {
    BwdInstance& I = L.inst[i];
    const PlanLayout::InstOff& o = L.inst_off[i];
    const FwdGroup& G = L.groups[o.group];
    I.E = G.E;
    I.V = G.V;
    I.ld = G.ld;
    I.Y = yreg + o.y;
    I.partial = (double*)(preg + o.partial);
    I.scale_tab = (double*)(sreg + o.scale);
    I.beta_hist = beta_hist;
    I.beta_z = o.beta == SIZE_MAX ? nullptr : (double*)(sreg + o.beta);
    I.oos_sum = o.oos_partial == SIZE_MAX ? nullptr : (double*)(sreg + o.oos_partial);
    I.oos_tab = o.oos_tab == SIZE_MAX ? nullptr : (void*)(sreg + o.oos_tab);
    I.oos_screen = o.oos_screen == SIZE_MAX ? nullptr : (void*)(sreg + o.oos_screen);
  }
  const FwdContract* dC = (const FwdContract*)put(L.contracts.data(), sizeof(FwdContract) * L.contracts.size());
  const FwdGroup* dG = (const FwdGroup*)put(L.groups.data(), sizeof(FwdGroup) * L.groups.size());
  p->d_inst = (BwdInstance*)put(L.inst.data(), sizeof(BwdInstance) * L.inst.size());
  const unsigned long long* dR = (const unsigned long long*)put(L.round_off.data(), sizeof(unsigned long long) * L.round_off.size());
  const uint32_t* dT = (const uint32_t*)put(L.cum_tiles.data(), sizeof(uint32_t) * L.cum_tiles.size());
  uint32_t zero = 0;
  const uint32_t* dA = (const uint32_t*)(L.active.empty() ? put(&zero, 4) : put(L.active.data(), sizeof(uint32_t) * L.active.size()));
  p->d_greeks = (GreekOut*)put(L.greeks.data(), sizeof(GreekOut) * L.greeks.size());
  const uint32_t* dQ = (const uint32_t*)put(L.req_info.data(), sizeof(uint32_t) * L.req_info.size());
  off = L.bytes_tables;
  p->d_state = take(L.bytes_state);
  p->state_bytes = L.bytes_state;
  p->d_ctl = (Control*)((char*)p->d_state + sizeof(BwdState) * L.inst.size());
  p->d_results = (BwdResult*)take(L.bytes_results);
  p->d_out = (DevResult*)take(L.bytes_out);
  LSMC_CUDA(cudaMemcpyAsync(base, blob.data(), blob.size(), cudaMemcpyHostToDevice, p->stream));

  p->fa.contracts = dC;
  p->fa.groups = dG;
  p->fa.n_contracts = (uint32_t)L.contracts.size();
  p->fa.n_blocks = L.fwd_blocks;
  p->fa.n0 = p->fa.n1 = 0;
  p->fa.row0 = 1;
  p->fa.ck_stride = L.opt.regen ? L.opt.ck_stride : 0;
  p->fa.store_rows = 1;
  p->fa.save_states = 0;
  p->fa.next_job = nullptr;
  p->fa.next_job_value = 0;
  p->fa.stream_xor = 0;
  p->fa.store_fmt = L.opt.store;
  // one seed for every contract: the Philox round keys as kernel parameters
  p->fa.uniform_key = 0;
  if (!L.contracts.empty()) {
    const uint64_t seed = L.contracts[0].seed;
    bool same = true;
    for (const auto& c : L.contracts) same = same && c.seed == seed;
    if (same) {
      uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
      for (int r = 0; r < 10; ++r) {
        p->fa.rk[2 * r] = k0;
        p->fa.rk[2 * r + 1] = k1;
        k0 += 0x9E3779B9u;  // the Weyl constants of the key schedule (Salmon et al.)
        k1 += 0xBB67AE85u;
      }
      p->fa.uniform_key = 1;
    }
  }
  p->ba.row0 = 1;
  p->ba.store_fmt = L.opt.store;
  p->ba.inst = p->d_inst;
  p->ba.state = (BwdState*)p->d_state;
  p->ba.results = p->d_results;
  p->ba.round_off = dR;
  p->ba.cum_tiles = dT;
  p->ba.active = dA;
  p->ba.ctl = p->d_ctl;
  p->ba.total_jobs = L.total_jobs;
  p->ba.req_count = (uint32_t*)(p->d_ctl + 1);
  p->ba.req_info = dQ;
  p->ba.greeks = p->d_greeks;
  p->ba.out_host = nullptr;  // per-request completion: set by the serving scheduler
  p->ba.flag_host = nullptr;
  // bound of each device-side wait: the context's limit (20 s unless set)
  const double limit_s = p->ctx ? p->ctx->wait_limit_s : 20.0;
  p->ba.timeout_ns = (unsigned long long)(limit_s * 1e9);
  p->ba.n_rounds = (uint32_t)L.active.size();
  p->ba.n_inst = (uint32_t)L.inst.size();
  const int occ = occupancy(p->ctx, prec, L.opt.basis, plan_ppt(L.opt), L.opt.store);
  const uint64_t cap = (uint64_t)occ * sm_count(p->ctx);
  p->bwd_grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(cap, L.total_jobs));
  p->h_out.resize(L.greeks.size());
  p->h_res.resize(L.n_results);
#ifdef LSMC_CHECKED
  {
    // the plan's allocation, and the caller's arrays of a stage call: paths
    // (rows 0..N, P apart) and the coefficient history (N x 6 doubles)
    CheckRanges c{};
    add_range(c, p->dev, L.total_bytes);
    const size_t N = L.contracts.empty() ? 0 : L.contracts[0].N;
    const size_t P = L.contracts.empty() ? 0 : L.contracts[0].P;
    add_range(c, ext_S, (N + 1) * P * real);
    add_range(c, ext_V, (N + 1) * P * real);
    add_range(c, beta_hist, N * 6 * sizeof(double));
    if (check_word(&c.err, &c.info) != LSMC_OK) return LSMC_ECUDA;
    p->chk = c;
    p->fa.chk = c;
    p->ba.chk = c;
  }
#endif
  return LSMC_OK;
}

int plan_alloc(lsmc_plan* p, bool use_arena, bool stream_ordered) {
  const size_t bytes = std::max<size_t>(p->L.total_bytes, 256);
  if (use_arena && p->ctx && p->ctx->arena.active()) {
    p->dev = (char*)p->ctx->arena.alloc(bytes);
    if (!p->dev) return LSMC_ENOMEM;
    p->alloc_kind = 1;
    return LSMC_OK;
  }
  if (p->ctx && p->ctx->dev_alloc) {
    p->dev = (char*)p->ctx->dev_alloc(bytes, p->ctx->alloc_user);
    if (!p->dev) return LSMC_ENOMEM;
    count_device_alloc();
    if ((uintptr_t)p->dev & 255) {  // the layout needs 256-byte alignment
      p->ctx->dev_free(p->dev, p->ctx->alloc_user);
      p->dev = nullptr;
      return LSMC_EINVAL;
    }
    p->alloc_kind = 3;
    return LSMC_OK;
  }
  if (stream_ordered) {
    LSMC_CUDA(cudaMallocAsync((void**)&p->dev, bytes, p->stream));
    count_device_alloc();
    p->alloc_kind = 2;
    return LSMC_OK;
  }
  LSMC_CUDA(cudaMalloc((void**)&p->dev, bytes));
  count_device_alloc();
  p->alloc_kind = 0;
  return LSMC_OK;
}

void plan_free(lsmc_plan* p) {
  if (!p) return;
  for (auto& e : p->ev)
    for (auto x : e) cudaEventDestroy(x);
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->dev) {
    if (p->alloc_kind == 1) {
      cudaStreamSynchronize(p->stream);
      p->ctx->arena.free(p->dev);
    } else if (p->alloc_kind == 2) {
      cudaFreeAsync(p->dev, p->stream);
    } else if (p->alloc_kind == 3) {
      cudaStreamSynchronize(p->stream);  // the callback may hand the memory out at once
      p->ctx->dev_free(p->dev, p->ctx->alloc_user);
    } else {
      cudaStreamSynchronize(p->stream);
      cudaFree(p->dev);
    }
  }
  delete p;
}

// requests of one plan share precision, scheme and basis
int plan_options(lsmc_ctx* ctx, const lsmc_request* reqs, size_t n, PlanOptions* o) {
  if (!reqs || n == 0) return LSMC_EINVAL;
  const int dprec = ctx ? ctx->precision : LSMC_FP64;
  const int dsch = ctx ? ctx->scheme : LSMC_SCHEME_QE;
  o->precision = resolve(ctx, reqs[0].precision, dprec);
  o->scheme = resolve(ctx, reqs[0].scheme, dsch);
  o->basis = reqs[0].basis;
  o->regen = (reqs[0].flags & LSMC_FLAG_REGENERATE) != 0;
  o->oos = (reqs[0].flags & LSMC_FLAG_OUT_OF_SAMPLE) != 0;
  const uint32_t store_flags = LSMC_FLAG_STORE_FP16 | LSMC_FLAG_STORE_BF16;
  o->store = (reqs[0].flags & LSMC_FLAG_STORE_FP16) ? kStoreF16
             : (reqs[0].flags & LSMC_FLAG_STORE_BF16) ? kStoreBF16 : kStoreNative;
  if (o->regen && o->oos) return LSMC_ENOTIMPL;
  for (size_t i = 0; i < n; ++i) {
    const int prec = resolve(ctx, reqs[i].precision, dprec);
    const int sch = resolve(ctx, reqs[i].scheme, dsch);
    int rc = validate_request(reqs[i], prec, sch);
    if (rc) return rc;
    if (prec != o->precision || sch != o->scheme || reqs[i].basis != o->basis)
      return LSMC_ENOTIMPL;
    // regenerate mode: one flag and one date grid for the whole plan
    if (((reqs[i].flags & LSMC_FLAG_REGENERATE) != 0) != o->regen) return LSMC_ENOTIMPL;
    if (((reqs[i].flags & LSMC_FLAG_OUT_OF_SAMPLE) != 0) != o->oos) return LSMC_ENOTIMPL;
    if ((reqs[i].flags & store_flags) != (reqs[0].flags & store_flags)) return LSMC_ENOTIMPL;
    if (o->regen && reqs[i].n_steps != reqs[0].n_steps) return LSMC_ENOTIMPL;
  }
  if (o->regen) {
    const uint32_t N = reqs[0].n_steps;
    uint32_t c = 1;
    while ((uint64_t)c * c < N) ++c;
    o->ck_stride = c;  // ceil(sqrt(N))
  }
  return LSMC_OK;
}

uint64_t tune_key(const lsmc_request* reqs, size_t n, const PlanOptions& o) {
  // sub-tiles (of the default shape) of the first round over all
  // instances, as a power of two
  const uint64_t tile0 = (uint64_t)backward_tile(o.precision, backward_ppt_default(o.precision));
  uint64_t tiles = 0;
  for (size_t i = 0; i < n; ++i) {
    std::vector<Scenario> sc;
    if (expand_scenarios(reqs[i], &sc) < 0) continue;
    tiles += (uint64_t)sc.size() * reqs[i].n_strikes * ((reqs[i].n_paths + tile0 - 1) / tile0);
  }
  uint64_t lg = 0;
  while ((2ull << lg) <= tiles) ++lg;
  return ((uint64_t)o.store << 48) | ((uint64_t)o.precision << 40) | ((uint64_t)o.basis << 32) | lg;
}

// Backward shape of a plan: autotuned if this kind of launch was tuned, else
// the precision's paths per thread and about four jobs per resident CTA in
// the busiest round; overrides (tuning sweeps) win.
void choose_shape(lsmc_ctx* ctx, const lsmc_request* reqs, size_t n, PlanOptions* o) {
  uint32_t tuned = 0;
  if (ctx) {
    auto it = ctx->tuned.find(tune_key(reqs, n, *o));
    if (it != ctx->tuned.end()) tuned = it->second;
  }
  o->ppt = tuned >> 16;
  if (ctx && ctx->ppt_override) o->ppt = ctx->ppt_override;
  const int ppt = plan_ppt(*o);
  const uint32_t ctas = (uint32_t)occupancy(ctx, o->precision, o->basis, ppt, o->store) *
                        (uint32_t)sm_count(ctx);
  o->sub = choose_sub(reqs, n, o->precision, ppt, ctas);
  if (tuned & 0xffffu) o->sub = tuned & 0xffffu;
  if (ctx && ctx->sub_override) o->sub = ctx->sub_override;
}

// subs (optional): the sub-tiles per job of each request, with paths per
// thread ppt, instead of the shape chosen for the whole plan.
int plan_create_on(lsmc_ctx* ctx, const lsmc_request* reqs, size_t n,
                   cudaStream_t stream, bool use_arena, lsmc_plan** out,
                   const std::vector<uint32_t>* subs = nullptr, uint32_t ppt = 0) {
  PlanOptions o;
  int rc = plan_options(ctx, reqs, n, &o);
  if (rc) return rc;
  std::unique_ptr<lsmc_plan> p(new (std::nothrow) lsmc_plan());
  if (!p) return LSMC_ENOMEM;
  p->ctx = ctx;
  p->stream = stream;
  if (subs && subs->size() == n) {
    o.ppt = ppt;
    o.sub_req = *subs;
  } else {
    choose_shape(ctx, reqs, n, &o);
  }
  rc = build_layout(reqs, n, o, &p->L);
  if (rc) return rc;
  rc = plan_alloc(p.get(), use_arena, false);
  if (rc) return rc;
  rc = plan_bind_and_upload(p.get(), nullptr, nullptr, nullptr);
  if (rc) { plan_free(p.release()); return rc; }
  *out = p.release();
  return LSMC_OK;
}

int plan_enqueue(lsmc_plan* p, bool timed = false) {
  const int prec = p->L.opt.precision;
  cudaEvent_t* ev = nullptr;
  if (timed) {
    if (p->ev_used == p->ev.size()) {
      std::array<cudaEvent_t, 5> e{};
      for (auto& x : e) LSMC_CUDA(cudaEventCreate(&x));
      p->ev.push_back(e);
    }
    ev = p->ev[p->ev_used++].data();
  }
  auto mark = [&](int i) { return ev ? cudaEventRecord(ev[i], p->stream) : cudaSuccess; };
  LSMC_CUDA(cudaMemsetAsync(p->d_state, 0, p->state_bytes, p->stream));
  LSMC_CUDA(mark(0));
  if (p->run_backward)
    LSMC_CUDA(launch_setup(p->d_inst, (uint32_t)p->L.inst.size(), p->stream CHK_ARG(p->chk)));
  LSMC_CUDA(mark(1));
  if (p->L.opt.regen && p->run_forward && p->run_backward) {
    // regenerate mode: one pass saving the states, then per segment of
    // dates (last first) the segment's rows simulated again and the
    // backward rounds whose dates lie in it; in the timing, the segments'
    // simulation counts with the backward pass
    FwdArgs f = p->fa;
    f.store_rows = 0;
    f.save_states = 1;
    LSMC_CUDA(launch_forward(f, prec, p->L.opt.scheme, p->stream));
    LSMC_CUDA(mark(2));
    const uint32_t N = p->L.contracts.empty() ? 0 : p->L.contracts[0].N;
    const uint32_t C = p->L.opt.ck_stride;
    const int occ = occupancy(p->ctx, prec, p->L.opt.basis, plan_ppt(p->L.opt), p->L.opt.store);
    const uint64_t cap = (uint64_t)occ * sm_count(p->ctx);
    for (int sgi = (int)p->L.n_segments - 1; sgi >= 0; --sgi) {
      const uint32_t d0 = (uint32_t)sgi * C, d1 = std::min<uint32_t>(N, d0 + C);
      // rounds r with regression date n = N - 1 - r in [d0, d1 - 1]
      const uint32_t r_lo = N - d1, r_hi = N - 1 - d0;  // inclusive
      const uint64_t nr = p->L.round_off.size() - 1;
      const uint64_t j0 = p->L.round_off[std::min<uint64_t>(r_lo, nr)];
      const uint64_t j1 = p->L.round_off[std::min<uint64_t>((uint64_t)r_hi + 1, nr)];
      FwdArgs g = p->fa;
      g.n0 = d0;
      g.n1 = d1;
      g.row0 = d0;
      g.store_rows = 1;
      g.save_states = 0;
      g.next_job = &p->d_ctl->next_job;
      g.next_job_value = j0;
      LSMC_CUDA(launch_forward(g, prec, p->L.opt.scheme, p->stream));
      if (j1 > j0) {
        BwdArgs b = p->ba;
        b.row0 = d0;
        b.total_jobs = j1;
        const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(cap, j1 - j0));
        LSMC_CUDA(launch_backward(b, prec, p->L.opt.basis, plan_ppt(p->L.opt), grid, p->stream));
      }
    }
    LSMC_CUDA(mark(3));
  } else {
    if (p->run_forward) LSMC_CUDA(launch_forward(p->fa, prec, p->L.opt.scheme, p->stream));
    LSMC_CUDA(mark(2));
    if (p->run_backward)
      LSMC_CUDA(launch_backward(p->ba, prec, p->L.opt.basis, plan_ppt(p->L.opt), p->bwd_grid,
                                p->stream));
    if (p->L.opt.oos && p->run_forward && p->run_backward) {
      // out of sample: the pricing paths (stream ^ 0x80000000) over the
      // regression paths' store, the policy applied to them, the estimator
      FwdArgs f = p->fa;
      f.stream_xor = 0x80000000u;
      LSMC_CUDA(launch_forward(f, prec, p->L.opt.scheme, p->stream));
      uint32_t max_p = 0;
      for (const auto& c : p->L.contracts) max_p = std::max(max_p, c.P);
      LSMC_CUDA(launch_oos(p->d_inst, (uint32_t)p->L.inst.size(), max_p, p->ba.state,
                           p->d_results, prec, p->L.opt.basis, p->L.opt.store,
                           p->stream CHK_ARG(p->chk)));
    }
    LSMC_CUDA(mark(3));
  }
  if (p->run_greeks)
    LSMC_CUDA(launch_greeks(p->d_greeks, p->d_results, (uint32_t)p->L.greeks.size(), p->d_out,
                            p->stream CHK_ARG(p->chk)));
  LSMC_CUDA(mark(4));
  return LSMC_OK;
}

int plan_launch(lsmc_plan* p, bool use_graph) {
  if (!use_graph || p->timing) return plan_enqueue(p, p->timing);
  if (!p->exec) {
    cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
    LSMC_CUDA(cudaStreamBeginCapture(p->stream, mode));
    int rc = plan_enqueue(p);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(p->stream, &g);
    if (rc) { if (g) cudaGraphDestroy(g); return rc; }
    LSMC_CUDA(e);
    p->graph = g;
    LSMC_CUDA(cudaGraphInstantiate(&p->exec, g, 0));
  }
  LSMC_CUDA(cudaGraphLaunch(p->exec, p->stream));
  return LSMC_OK;
}

int plan_collect(lsmc_plan* p, lsmc_result* outs) {
  Control ctl{};
  LSMC_CUDA(cudaMemcpyAsync(&ctl, p->d_ctl, sizeof(Control), cudaMemcpyDeviceToHost, p->stream));
  if (!p->h_res.empty())
    LSMC_CUDA(cudaMemcpyAsync(p->h_res.data(), p->d_results, sizeof(BwdResult) * p->h_res.size(),
                              cudaMemcpyDeviceToHost, p->stream));
  if (!p->h_out.empty())
    LSMC_CUDA(cudaMemcpyAsync(p->h_out.data(), p->d_out, sizeof(DevResult) * p->h_out.size(),
                              cudaMemcpyDeviceToHost, p->stream));
  LSMC_CUDA(cudaStreamSynchronize(p->stream));
  if (ctl.error == kDevErrTimeout) return LSMC_ETIMEOUT;
  if (ctl.error) return LSMC_ECUDA;
  double itm = 0;
  for (const auto& r : p->h_res) {
    if (p->run_backward && !r.done) return LSMC_ECUDA;
    itm += r.itm;
  }
  p->itm = (uint64_t)itm;
  if (outs) std::memcpy(outs, p->h_out.data(), sizeof(DevResult) * p->h_out.size());
  return LSMC_OK;
}

// ---- serving ---------------------------------------------------------------------
void finish_ticket(lsmc_ctx* ctx, Ticket* t, int status) {
  t->status = status;
  t->t_done = now_s() - ctx->t0;
  ctx->done_cv.notify_all();
}

// Requests admitted together share one plan (one launch of each kernel).
constexpr size_t kMaxBatch = 64;  // default and upper limit of lsmc_config.max_batch
constexpr uint32_t kMaxServeSub = 32;

// Arms per-request completion for the plan of an idle slot: host-mapped room
// for the plan's results and its requests' flags (grown when too small), the
// flags cleared, the backward pass pointed at them.  Out-of-sample plans
// price after the backward pass and finish with their batch.
int arm_early_results(Slot& sl, lsmc_plan* p, size_t n_req) {
  if (p->L.opt.oos) return LSMC_OK;
  const size_t n_out = p->L.greeks.size();
  if (n_out > sl.cap_out) {
    if (sl.map_out) cudaFreeHost(sl.map_out);
    sl.map_out = nullptr;
    sl.cap_out = 0;
    const size_t cap = std::max<size_t>(n_out, 4 * kMaxBatch);
    LSMC_CUDA(cudaHostAlloc((void**)&sl.map_out, cap * sizeof(DevResult), cudaHostAllocMapped));
    sl.cap_out = cap;
  }
  if (n_req > sl.cap_req) {
    if (sl.map_flag) cudaFreeHost(sl.map_flag);
    sl.map_flag = nullptr;
    sl.cap_req = 0;
    const size_t cap = std::max<size_t>(n_req, kMaxBatch);
    LSMC_CUDA(cudaHostAlloc((void**)&sl.map_flag, cap * sizeof(uint32_t), cudaHostAllocMapped));
    sl.cap_req = cap;
  }
  std::memset(sl.map_flag, 0, n_req * sizeof(uint32_t));
  void* d_out = nullptr;
  void* d_flag = nullptr;
  LSMC_CUDA(cudaHostGetDevicePointer(&d_out, sl.map_out, 0));
  LSMC_CUDA(cudaHostGetDevicePointer(&d_flag, sl.map_flag, 0));
  p->ba.out_host = (DevResult*)d_out;
  p->ba.flag_host = (uint32_t*)d_flag;
#ifdef LSMC_CHECKED
  add_range(p->ba.chk, d_out, n_out * sizeof(DevResult));
  add_range(p->ba.chk, d_flag, n_req * sizeof(uint32_t));
#endif
  return LSMC_OK;
}

void scheduler_loop(lsmc_ctx* ctx) {
  cudaSetDevice(ctx->device);
  std::unique_lock<std::mutex> lk(ctx->mu);
  while (!ctx->stop) {
    bool progress = false;
    for (size_t s = 0; s < ctx->slots.size(); ++s) {
      Slot& sl = ctx->slots[s];
      if (sl.batch.empty()) continue;
      // requests whose results the device has handed over already
      if (sl.plan && sl.plan->ba.flag_host) {
        size_t off = 0;
        for (size_t i = 0; i < sl.batch.size(); ++i) {
          Ticket* t = sl.batch[i];
          if (t && ((volatile uint32_t*)sl.map_flag)[i] != 0u) {
            std::atomic_thread_fence(std::memory_order_acquire);
            t->results.resize(sl.nk[i]);
            std::memcpy(t->results.data(), sl.map_out + off, sizeof(lsmc_result) * sl.nk[i]);
            finish_ticket(ctx, t, LSMC_OK);
            sl.batch[i] = nullptr;
            progress = true;
          }
          off += sl.nk[i];
        }
      }
      // the rest of a batch finishes with its launch
      const cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaErrorNotReady) continue;
      int rc = q == cudaSuccess ? LSMC_OK : LSMC_ECUDA;
      std::vector<lsmc_result> all;
      if (rc == LSMC_OK) {
        all.resize(sl.plan->h_out.size());
        rc = plan_collect(sl.plan, all.data());
      }
      size_t off = 0;
      for (size_t i = 0; i < sl.batch.size(); ++i) {
        Ticket* t = sl.batch[i];
        const size_t k = sl.nk[i];
        if (t) {
          if (rc == LSMC_OK && off + k <= all.size())
            t->results.assign(all.begin() + off, all.begin() + off + k);
          finish_ticket(ctx, t, rc);
        }
        off += k;
      }
      plan_free(sl.plan);
      sl.plan = nullptr;
      sl.batch.clear();
      sl.nk.clear();
      progress = true;
    }
    // admissions, first come first served: the oldest pending request and
    // the pending requests right behind it that can share its launch (same
    // precision, scheme, basis, paths per thread and flags) while the workspace
    // has room for all of them
    while (!ctx->pending.empty()) {
      int free_slot = -1;
      for (size_t s = 0; s < ctx->slots.size(); ++s)
        if (ctx->slots[s].batch.empty()) { free_slot = (int)s; break; }
      if (free_slot < 0) break;
      Ticket* t0 = ctx->pending.front();
      const size_t room = ctx->arena.largest_free();
      if (room < t0->footprint) break;  // wait for memory
      std::vector<Ticket*> batch{t0};
      size_t need = t0->footprint;
      for (size_t i = 1; i < ctx->pending.size() && batch.size() < ctx->max_batch; ++i) {
        Ticket* t = ctx->pending[i];
        if (t->precision != t0->precision || t->scheme != t0->scheme ||
            t->basis != t0->basis || t->ppt != t0->ppt || t->req.flags != t0->req.flags ||
            ((t->req.flags & LSMC_FLAG_REGENERATE) && t->req.n_steps != t0->req.n_steps) ||
            need + t->footprint > room)
          break;
        batch.push_back(t);
        need += t->footprint;
      }
      // The batch leaves the queue and reserves the slot; its plan is built
      // and launched without the context lock, so submit, poll and wait
      // callers are not held up by validation, layout and the table upload
      // (only this thread admits or completes batches).
      Slot& sl = ctx->slots[free_slot];
      ctx->pending.erase(ctx->pending.begin(), ctx->pending.begin() + batch.size());
      const double t_admit = now_s() - ctx->t0;
      for (Ticket* t : batch) {
        t->t_admit = t_admit;
        t->slot = free_slot;
      }
      sl.batch = batch;
      sl.plan = nullptr;
      const uint32_t ppt = t0->ppt;
      const double share =
          ctx->serve_share > 0.0 ? ctx->serve_share : 1.0 / (double)ctx->slots.size();
      lk.unlock();
      lsmc_plan* p = nullptr;
      int rc = LSMC_ENOMEM;
      size_t take = batch.size();
      while (take > 0) {
        std::vector<lsmc_request> reqs;
        std::vector<uint32_t> subs;
        for (size_t i = 0; i < take; ++i) {
          reqs.push_back(batch[i]->req);
          subs.push_back(batch[i]->sub);
        }
        rc = plan_create_on(ctx, reqs.data(), reqs.size(), sl.stream, true, &p, &subs, ppt);
        if (rc != LSMC_ENOMEM || take == 1) break;
        take /= 2;  // fragmentation: a smaller batch
      }
      // the batch's persistent backward grid: its share of the device
      if (rc == LSMC_OK && share < 1.0) {
        const int occ = occupancy(ctx, p->L.opt.precision, p->L.opt.basis, plan_ppt(p->L.opt),
                                  p->L.opt.store);
        const int part = (int)std::ceil(share * occ * sm_count(ctx));
        p->bwd_grid = std::max(1, std::min(p->bwd_grid, part));
      }
      // without host-mapped room the batch's requests finish together
      if (rc == LSMC_OK && arm_early_results(sl, p, take) != LSMC_OK) {
        p->ba.out_host = nullptr;
        p->ba.flag_host = nullptr;
      }
      if (rc == LSMC_OK) rc = plan_launch(p, false);
      if (rc == LSMC_OK && cudaEventRecord(sl.done, sl.stream) != cudaSuccess) rc = LSMC_ECUDA;
      lk.lock();
      // requests that did not fit go back to the front of the queue, in order
      const size_t back = rc == LSMC_ENOMEM ? 0 : take;
      if (back < batch.size()) {
        ctx->pending.insert(ctx->pending.begin(), batch.begin() + back, batch.end());
        for (size_t i = back; i < batch.size(); ++i) {
          batch[i]->t_admit = 0;
          batch[i]->slot = -1;
        }
        batch.resize(back);
      }
      sl.batch.clear();
      if (rc == LSMC_ENOMEM) break;  // retry once others finish
      if (rc != LSMC_OK) {
        if (p) plan_free(p);
        for (Ticket* t : batch) finish_ticket(ctx, t, rc);
      } else {
        sl.plan = p;
        sl.batch = batch;
        sl.nk.clear();
        for (Ticket* t : batch) sl.nk.push_back(t->req.n_strikes);
      }
      progress = true;
    }
    bool inflight = false;
    for (const auto& sl : ctx->slots) inflight |= !sl.batch.empty();
    if (!inflight && ctx->pending.empty()) {
      ctx->cv.wait(lk, [&] { return ctx->stop || !ctx->pending.empty(); });
    } else if (!progress) {
      ctx->cv.wait_for(lk, std::chrono::microseconds(50));
    }
  }
}

int start_scheduler(lsmc_ctx* ctx) {
  if (ctx->sched_started) return LSMC_OK;
  if (!ctx->arena.active()) {
    size_t budget = ctx->hbm_budget;
    if (budget == 0) {
      size_t fr = 0, tot = 0;
      LSMC_CUDA(cudaMemGetInfo(&fr, &tot));
      budget = std::min<size_t>(fr / 4 * 3, (size_t)64 << 30);
    }
    if (ctx->dev_alloc) {
      ctx->own_arena_mem = ctx->dev_alloc(budget, ctx->alloc_user);
      if (!ctx->own_arena_mem) return LSMC_ENOMEM;
      count_device_alloc();
      if ((uintptr_t)ctx->own_arena_mem & 255) {
        ctx->dev_free(ctx->own_arena_mem, ctx->alloc_user);
        ctx->own_arena_mem = nullptr;
        return LSMC_EINVAL;
      }
    } else {
      LSMC_CUDA(cudaMalloc(&ctx->own_arena_mem, budget));
      count_device_alloc();
    }
    ctx->arena.reset(ctx->own_arena_mem, budget);
  }
  // a later call after a failure here keeps what an earlier one created
  ctx->slots.resize(ctx->max_inflight);
  for (auto& s : ctx->slots) {
    if (!s.stream) LSMC_CUDA(cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking));
    if (!s.done) LSMC_CUDA(cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming));
  }
  ctx->sched = std::thread(scheduler_loop, ctx);
  ctx->sched_started = true;
  return LSMC_OK;
}

lsmc_request default_request(const lsmc_heston* m, const lsmc_contract* c, uint32_t P,
                             uint32_t N, int32_t basis, const lsmc_bumps* b, uint64_t seed) {
  lsmc_request q{};
  q.model = *m;
  q.type = c->type;
  q.style = c->style;
  q.T = c->T;
  q.strikes = &c->K;
  q.n_strikes = 1;
  q.n_paths = P;
  q.n_steps = N;
  q.basis = basis;
  q.precision = -1;
  q.scheme = -1;
  if (b) q.bumps = *b;
  q.seed = seed;
  q.stream_id = 0;
  return q;
}

}  // namespace

extern "C" {

const char* lsmc_strerror(int s) {
  switch (s) {
    case LSMC_OK: return "ok";
    case LSMC_PENDING: return "pending";
    case LSMC_EINVAL: return "invalid argument";
    case LSMC_ENOMEM: return "out of device or workspace memory";
    case LSMC_EBUSY: return "request queue full";
    case LSMC_ETIMEOUT: return "bounded device wait expired";
    case LSMC_ECUDA: return "CUDA runtime error";
    case LSMC_ENOTIMPL: return "not supported";
    case LSMC_ENOTFOUND: return "unknown ticket";
    case LSMC_ENODEV: return "no usable CUDA device";
    default: return "unknown status";
  }
}

int lsmc_abi_version(void) { return LSMC_ABI_VERSION; }

int lsmc_device_allocations(uint64_t* count) {
  if (!count) return LSMC_EINVAL;
  *count = g_device_allocs.load(std::memory_order_relaxed);
  return LSMC_OK;
}

int lsmc_create(lsmc_ctx** out, const lsmc_config* cfg) {
  if (!out) return LSMC_EINVAL;
  *out = nullptr;
  lsmc_config c{};
  if (cfg) c = *cfg;
  if (c.precision != LSMC_FP64 && c.precision != LSMC_MIXED && c.precision != LSMC_DF)
    return LSMC_EINVAL;
  if (c.scheme != LSMC_SCHEME_QE && c.scheme != LSMC_SCHEME_FT_EULER) return LSMC_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) return LSMC_ENODEV;
  if (c.device < 0 || c.device >= ndev) return LSMC_EINVAL;
  LSMC_CUDA(cudaSetDevice(c.device));
  lsmc_ctx* ctx = new (std::nothrow) lsmc_ctx();
  if (!ctx) return LSMC_ENOMEM;
  ctx->device = c.device;
  ctx->precision = c.precision;
  ctx->scheme = c.scheme;
  ctx->hbm_budget = (size_t)c.hbm_budget;
  ctx->max_inflight = c.max_inflight ? c.max_inflight : 8;
  ctx->queue_capacity = c.queue_capacity ? c.queue_capacity : 4096;
  ctx->max_batch = c.max_batch > 0 ? std::min<uint32_t>((uint32_t)c.max_batch, kMaxBatch)
                                   : (uint32_t)kMaxBatch;
  ctx->t0 = now_s();
  if (cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete ctx;
    return LSMC_ECUDA;
  }
  ctx->stream = ctx->own_stream;
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, c.device);
  *out = ctx;
  return LSMC_OK;
}

void lsmc_destroy(lsmc_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  {
    std::unique_lock<std::mutex> lk(ctx->mu);
    ctx->stop = true;
  }
  ctx->cv.notify_all();
  if (ctx->sched.joinable()) ctx->sched.join();
  for (auto& s : ctx->slots) {
    if (s.stream) cudaStreamSynchronize(s.stream);
    if (s.plan) plan_free(s.plan);
    s.plan = nullptr;
    s.batch.clear();
  }
  for (auto& kv : ctx->tickets) delete kv.second;
  for (auto& s : ctx->slots) {
    if (s.done) cudaEventDestroy(s.done);
    if (s.stream) cudaStreamDestroy(s.stream);
    if (s.map_out) cudaFreeHost(s.map_out);
    if (s.map_flag) cudaFreeHost(s.map_flag);
  }
  if (ctx->own_stream) {
    cudaStreamSynchronize(ctx->own_stream);
    cudaStreamDestroy(ctx->own_stream);
  }
  if (ctx->own_arena_mem) {
    cudaDeviceSynchronize();
    if (ctx->dev_free) ctx->dev_free(ctx->own_arena_mem, ctx->alloc_user);
    else cudaFree(ctx->own_arena_mem);
  }
  delete ctx;
}

int lsmc_set_stream(lsmc_ctx* ctx, void* s) {
  if (!ctx) return LSMC_EINVAL;
  ctx->stream = s ? (cudaStream_t)s : ctx->own_stream;
  return LSMC_OK;
}

int lsmc_set_allocator(lsmc_ctx* ctx, void* (*alloc)(size_t, void*),
                       void (*release)(void*, void*), void* user) {
  if (!ctx || (alloc == nullptr) != (release == nullptr)) return LSMC_EINVAL;
  std::lock_guard<std::mutex> g(ctx->mu);
  if (ctx->own_arena_mem || ctx->sched_started) return LSMC_EBUSY;
  ctx->dev_alloc = alloc;
  ctx->dev_free = release;
  ctx->alloc_user = user;
  return LSMC_OK;
}

int lsmc_set_wait_limit(lsmc_ctx* ctx, double seconds) {
  if (!ctx || !(seconds >= 0.0) || !(seconds <= 3600.0)) return LSMC_EINVAL;
  std::lock_guard<std::mutex> g(ctx->mu);
  ctx->wait_limit_s = seconds;
  return LSMC_OK;
}

int lsmc_set_backward_shape(lsmc_ctx* ctx, uint32_t sub, uint32_t ppt) {
  const uint32_t count = sub & ~LSMC_SUB_ITM_HALF;
  if (!ctx || count > kMaxSub || (count == 0 && sub != 0) ||
      !(ppt == 0 || ppt == 2 || ppt == 4 || ppt == 8))
    return LSMC_EINVAL;
  std::lock_guard<std::mutex> g(ctx->mu);
  ctx->sub_override = sub;
  ctx->ppt_override = ppt;
  return LSMC_OK;
}

int lsmc_set_serving_share(lsmc_ctx* ctx, double share) {
  if (!ctx || !(share >= 0.0 && share <= 1.0)) return LSMC_EINVAL;
  std::lock_guard<std::mutex> g(ctx->mu);
  ctx->serve_share = share;
  return LSMC_OK;
}

int lsmc_set_workspace(lsmc_ctx* ctx, void* ptr, size_t bytes) {
  if (!ctx || !ptr || bytes < 4096 || ((uintptr_t)ptr & 255)) return LSMC_EINVAL;
  std::lock_guard<std::mutex> g(ctx->mu);
  if (ctx->arena.active() && ctx->arena.used()) return LSMC_EBUSY;
  if (ctx->own_arena_mem) return LSMC_EBUSY;
  ctx->arena.reset(ptr, bytes);
  ctx->user_workspace = true;
  return LSMC_OK;
}

int lsmc_request_footprint(const lsmc_ctx* ctx, const lsmc_request* req, size_t* bytes) {
  if (!req || !bytes) return LSMC_EINVAL;
  PlanOptions o;
  int rc = plan_options(const_cast<lsmc_ctx*>(ctx), req, 1, &o);
  if (rc) return rc;
  PlanLayout L;
  rc = build_layout(req, 1, o, &L);
  if (rc) return rc;
  *bytes = align256(L.total_bytes);
  return LSMC_OK;
}

int lsmc_plan_layout_info(const lsmc_ctx* ctx, const lsmc_request* reqs, size_t n, uint32_t sub,
                          uint32_t ppt, lsmc_plan_info* info) {
  const uint32_t count = sub & ~LSMC_SUB_ITM_HALF;
  if (!reqs || !n || !info || count < 1 || count > kMaxSub ||
      !(ppt == 0 || ppt == 2 || ppt == 4 || ppt == 8))
    return LSMC_EINVAL;
  PlanOptions o;
  int rc = plan_options(const_cast<lsmc_ctx*>(ctx), reqs, n, &o);
  if (rc) return rc;
  o.sub = sub;
  o.ppt = ppt;
  PlanLayout L;
  rc = build_layout(reqs, n, o, &L);
  if (rc) return rc;
  *info = lsmc_plan_info{};
  info->generated_path_steps = L.generated_path_steps;
  info->lsmc_path_steps = L.lsmc_path_steps;
  info->backward_jobs = L.total_jobs;
  info->device_bytes = L.total_bytes;
  info->kernels_per_launch = 4;
  info->n_results = (uint32_t)L.greeks.size();
  info->n_instances = (uint32_t)L.inst.size();
  info->n_groups = (uint32_t)L.groups.size();
  info->h2d_bytes = L.bytes_tables;
  return LSMC_OK;
}

int lsmc_plan_create(lsmc_ctx* ctx, const lsmc_request* reqs, size_t n, lsmc_plan** out) {
  if (!ctx || !out) return LSMC_EINVAL;
  *out = nullptr;
  cudaSetDevice(ctx->device);
  return plan_create_on(ctx, reqs, n, ctx->stream, ctx->user_workspace, out);
}

int lsmc_plan_launch(lsmc_plan* p, int32_t use_graph) {
  if (!p) return LSMC_EINVAL;
  return plan_launch(p, use_graph != 0);
}

int lsmc_plan_fetch(lsmc_plan* p, lsmc_result* outs) {
  if (!p || !outs) return LSMC_EINVAL;
  return plan_collect(p, outs);
}

int lsmc_plan_fetch_scenarios(lsmc_plan* p, double* prices, uint32_t* near_ties,
                              size_t n_results) {
  if (!p || !prices || n_results != p->L.greeks.size()) return LSMC_EINVAL;
  if (!p->h_res.empty())
    LSMC_CUDA(cudaMemcpyAsync(p->h_res.data(), p->d_results, sizeof(BwdResult) * p->h_res.size(),
                              cudaMemcpyDeviceToHost, p->stream));
  LSMC_CUDA(cudaStreamSynchronize(p->stream));
  const double nan = std::nan("");
  for (size_t k = 0; k < n_results; ++k)
    for (int s = 0; s < kScCount; ++s) {
      const int32_t i = p->L.greeks[k].res[s];
      const bool have = i >= 0 && (size_t)i < p->h_res.size();
      prices[k * kScCount + s] = have ? p->h_res[i].price : nan;
      if (near_ties) near_ties[k * kScCount + s] = have ? (uint32_t)p->h_res[i].ties : 0u;
    }
  return LSMC_OK;
}

int lsmc_plan_device_results(lsmc_plan* p, void** ptr, size_t* count) {
  if (!p || !ptr || !count) return LSMC_EINVAL;
  *ptr = p->d_out;
  *count = p->L.greeks.size();
  return LSMC_OK;
}

int lsmc_plan_get_info(const lsmc_plan* p, lsmc_plan_info* info) {
  if (!p || !info) return LSMC_EINVAL;
  info->generated_path_steps = p->L.generated_path_steps;
  info->lsmc_path_steps = p->L.lsmc_path_steps;
  info->backward_jobs = p->L.total_jobs;
  info->device_bytes = p->L.total_bytes;
  info->kernels_per_launch = (p->run_backward ? 2 : 0) + (p->run_forward ? 1 : 0) + (p->run_greeks ? 1 : 0);
  info->n_results = (uint32_t)p->L.greeks.size();
  info->n_instances = (uint32_t)p->L.inst.size();
  info->n_groups = (uint32_t)p->L.groups.size();
  info->itm_path_steps = p->itm;
  info->h2d_bytes = p->L.bytes_tables;
  info->d2h_bytes = sizeof(Control) + sizeof(BwdResult) * p->h_res.size() +
                    sizeof(DevResult) * p->h_out.size();
  return LSMC_OK;
}

int lsmc_plan_set_timing(lsmc_plan* p, int32_t enable) {
  if (!p) return LSMC_EINVAL;
  p->timing = enable != 0;
  return LSMC_OK;
}

int lsmc_plan_kernel_times(lsmc_plan* p, double ms[4], uint32_t* launches) {
  if (!p || !ms) return LSMC_EINVAL;
  for (int i = 0; i < 4; ++i) ms[i] = 0.0;
  if (p->ev_used) LSMC_CUDA(cudaEventSynchronize(p->ev[p->ev_used - 1][4]));
  for (size_t k = 0; k < p->ev_used; ++k)
    for (int i = 0; i < 4; ++i) {
      float t = 0.f;
      LSMC_CUDA(cudaEventElapsedTime(&t, p->ev[k][i], p->ev[k][i + 1]));
      ms[i] += t;
    }
  if (launches) *launches = (uint32_t)p->ev_used;
  p->ev_used = 0;
  return LSMC_OK;
}

void lsmc_plan_destroy(lsmc_plan* p) { plan_free(p); }

int lsmc_price_request(lsmc_ctx* ctx, const lsmc_request* req, lsmc_result* outs) {
  if (!ctx || !req || !outs) return LSMC_EINVAL;
  lsmc_plan* p = nullptr;
  int rc = lsmc_plan_create(ctx, req, 1, &p);
  if (rc) return rc;
  rc = plan_launch(p, false);
  if (rc == LSMC_OK) rc = plan_collect(p, outs);
  plan_free(p);
  return rc;
}

int lsmc_price_greeks(lsmc_ctx* ctx, const lsmc_heston* m, const lsmc_contract* c,
                      uint32_t P, uint32_t N, int32_t basis, const lsmc_bumps* b,
                      uint64_t seed, lsmc_result* out) {
  if (!ctx || !m || !c || !b || !out) return LSMC_EINVAL;
  lsmc_request q = default_request(m, c, P, N, basis, b, seed);
  return lsmc_price_request(ctx, &q, out);
}

int lsmc_price_book(lsmc_ctx* ctx, const lsmc_request* reqs, size_t n, lsmc_result* outs) {
  if (!ctx || !reqs || !n || !outs) return LSMC_EINVAL;
  lsmc_plan* p = nullptr;
  int rc = lsmc_plan_create(ctx, reqs, n, &p);
  if (rc) return rc;
  rc = plan_launch(p, true);
  if (rc == LSMC_OK) rc = plan_collect(p, outs);
  plan_free(p);
  return rc;
}

int lsmc_price_bounds(lsmc_ctx* ctx, const lsmc_request* req, uint32_t n_outer,
                      uint32_t n_inner, lsmc_bounds* outs) {
  if (!ctx || !req || !outs) return LSMC_EINVAL;
  if (req->style != LSMC_AMERICAN || n_outer == 0 || n_inner == 0 ||
      n_outer > req->n_paths || req->n_strikes == 0 ||
      req->n_strikes > (uint32_t)kMaxDualStrikes ||
      (uint64_t)n_outer * req->n_steps + 1 > 0x7fffffffull)
    return LSMC_EINVAL;
  if (req->flags & LSMC_FLAG_REGENERATE) return LSMC_ENOTIMPL;
  // the base scenario only, with the policy's coefficients kept and priced
  // out of sample: the lower bound
  lsmc_request q = *req;
  q.bumps.greek_mask = 0;
  q.flags |= LSMC_FLAG_OUT_OF_SAMPLE;
  lsmc_plan* p = nullptr;
  int rc = lsmc_plan_create(ctx, &q, 1, &p);
  if (rc) return rc;
  const uint32_t nk = q.n_strikes, N = q.n_steps;
  std::vector<lsmc_result> res(nk);
  rc = plan_launch(p, false);
  if (rc == LSMC_OK) rc = plan_collect(p, res.data());
  if (rc) { plan_free(p); return rc; }
  const PlanLayout& L = p->L;
  const int prec = L.opt.precision;
  DualArgs a{};
  a.inst = p->d_inst;
  for (uint32_t k = 0; k < nk; ++k) {
    const int32_t slot = L.greeks[k].res[kScBase];
    for (size_t i = 0; i < L.inst.size(); ++i)
      if ((int32_t)L.inst[i].out_index == slot) a.inst_of_strike[k] = (uint32_t)i;
  }
  a.group = L.groups[L.contracts[0].group0];
  a.seed = q.seed;
  a.stream = q.stream_id;
  a.type = q.type;
  a.N = N;
  a.n_outer = n_outer;
  a.n_inner = n_inner;
  a.n_strikes = nk;
  const size_t real = value_bytes(prec);
  const size_t bx = align256((size_t)(N + 1) * n_outer * real);
  const size_t bq = align256((size_t)nk * n_outer * N * 8);
  const size_t bd = align256((size_t)nk * n_outer * 8);
  const size_t bti = align256((size_t)n_outer * N * 4);
  const size_t btm = align256((size_t)nk * n_outer * 4);
  const size_t bo = align256((size_t)nk * kDualOut * 8);
  const size_t total = 2 * bx + bq + 2 * bd + bti + btm + bo;
  char* mem = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  std::vector<double> o((size_t)nk * kDualOut, 0.0);
  float ms = 0.0f;
  cudaError_t ce = cudaSuccess;
  if (ctx->dev_alloc) {
    mem = (char*)ctx->dev_alloc(total, ctx->alloc_user);
    if (!mem) { plan_free(p); return LSMC_ENOMEM; }
    count_device_alloc();
    if ((uintptr_t)mem & 255) {  // the sub-buffers are laid out on 256-byte boundaries
      ctx->dev_free(mem, ctx->alloc_user);
      plan_free(p);
      return LSMC_EINVAL;
    }
  } else {
    ce = cudaMallocAsync((void**)&mem, total, p->stream);
    if (ce == cudaSuccess) count_device_alloc();
  }
  if (ce == cudaSuccess) {
    char* c = mem;
    a.X = c; c += bx;
    a.V = c; c += bx;
    a.Q = (double*)c; c += bq;
    a.dmax = (double*)c; c += bd;
    a.piN = (double*)c; c += bd;
    a.inner_ties = (uint32_t*)c; c += bti;
    a.max_ties = (uint32_t*)c; c += btm;
    a.out = (double*)c;
#ifdef LSMC_CHECKED
    a.chk = p->chk;
    add_range(a.chk, mem, total);
#endif
    if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce == cudaSuccess) ce = cudaEventRecord(e0, p->stream);
    if (ce == cudaSuccess) ce = launch_dual(a, prec, L.opt.scheme, L.opt.basis, p->stream);
    if (ce == cudaSuccess) ce = cudaEventRecord(e1, p->stream);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(o.data(), a.out, o.size() * 8, cudaMemcpyDeviceToHost, p->stream);
    const cudaError_t se = cudaStreamSynchronize(p->stream);
    if (ctx->dev_free) ctx->dev_free(mem, ctx->alloc_user);
    else cudaFreeAsync(mem, p->stream);
    if (ce == cudaSuccess) ce = se;
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  plan_free(p);
  if (ce != cudaSuccess) return cuda_status(ce);
  double ties = 0.0;
  for (uint32_t k = 0; k < nk; ++k) ties += o[(size_t)k * kDualOut + 4];
  for (uint32_t k = 0; k < nk; ++k) {
    lsmc_bounds& b = outs[k];
    const double* ok = o.data() + (size_t)k * kDualOut;
    b.lower = res[k].price;
    b.lower_se = res[k].price_se;
    b.upper = ok[0];
    b.upper_se = ok[1];
    b.martingale_end = ok[2];
    b.martingale_end_se = ok[3];
    b.dual_ms = ms;
    b.n_near_ties = res[k].n_near_ties + (uint32_t)ties;
    b.status = res[k].status;
  }
  return LSMC_OK;
}

// ---- serving -------------------------------------------------------------------
int lsmc_submit(lsmc_ctx* ctx, const lsmc_request* req, uint64_t* ticket) {
  if (!ctx || !req || !ticket) return LSMC_EINVAL;
  PlanOptions o;
  int rc = plan_options(ctx, req, 1, &o);
  if (rc) return rc;
  size_t fp = 0;
  rc = lsmc_request_footprint(ctx, req, &fp);
  if (rc) return rc;
  std::unique_lock<std::mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  rc = start_scheduler(ctx);
  if (rc) return rc;
  if (fp > ctx->arena.capacity()) return LSMC_ENOMEM;
  if (ctx->pending.size() >= ctx->queue_capacity) return LSMC_EBUSY;
  Ticket* t = new (std::nothrow) Ticket();
  if (!t) return LSMC_ENOMEM;
  t->id = ctx->next_ticket++;
  t->req = *req;
  t->strikes.assign(req->strikes, req->strikes + req->n_strikes);
  t->req.strikes = t->strikes.data();
  t->footprint = fp;
  t->precision = o.precision;
  t->scheme = o.scheme;
  t->basis = o.basis;
  // serving shape, a function of the request alone (so its result does not
  // depend on the batch it runs in): the precision's paths per thread and
  // about four jobs per regression and date, at most kMaxServeSub sub-tiles
  o.ppt = ctx->ppt_override;
  t->ppt = (uint32_t)plan_ppt(o);
  const uint32_t tile = (uint32_t)backward_tile(o.precision, (int)t->ppt);
  const uint32_t tiles = (req->n_paths + tile - 1) / tile;
  t->sub = ctx->sub_override ? ctx->sub_override
                             : std::min<uint32_t>(kMaxServeSub, std::max<uint32_t>(1, (tiles + 3) / 4));
  t->t_submit = now_s() - ctx->t0;
  ctx->tickets[t->id] = t;
  ctx->pending.push_back(t);
  *ticket = t->id;
  lk.unlock();
  ctx->cv.notify_all();
  return LSMC_OK;
}

static int take_result(lsmc_ctx* ctx, std::map<uint64_t, Ticket*>::iterator it, lsmc_result* outs) {
  Ticket* t = it->second;
  const int st = t->status;
  ctx->history[t->id] = {t->t_submit, t->t_admit, t->t_done};
  while (ctx->history.size() > (1u << 20)) ctx->history.erase(ctx->history.begin());
  if (st == LSMC_OK && outs)
    std::memcpy(outs, t->results.data(), sizeof(lsmc_result) * t->results.size());
  ctx->tickets.erase(it);
  delete t;
  return st;
}

int lsmc_poll(lsmc_ctx* ctx, uint64_t ticket, lsmc_result* outs) {
  if (!ctx) return LSMC_EINVAL;
  std::lock_guard<std::mutex> g(ctx->mu);
  auto it = ctx->tickets.find(ticket);
  if (it == ctx->tickets.end()) return LSMC_ENOTFOUND;
  if (it->second->status == LSMC_PENDING) return LSMC_PENDING;
  return take_result(ctx, it, outs);
}

int lsmc_wait(lsmc_ctx* ctx, uint64_t ticket, lsmc_result* outs, double timeout_s) {
  if (!ctx) return LSMC_EINVAL;
  std::unique_lock<std::mutex> lk(ctx->mu);
  auto pred = [&] {
    auto it = ctx->tickets.find(ticket);
    return it == ctx->tickets.end() || it->second->status != LSMC_PENDING;
  };
  if (timeout_s < 0) {
    ctx->done_cv.wait(lk, pred);
  } else {
    ctx->done_cv.wait_for(lk, std::chrono::duration<double>(timeout_s), pred);
  }
  auto it = ctx->tickets.find(ticket);
  if (it == ctx->tickets.end()) return LSMC_ENOTFOUND;
  if (it->second->status == LSMC_PENDING) return LSMC_PENDING;
  return take_result(ctx, it, outs);
}

int lsmc_ticket_times(lsmc_ctx* ctx, uint64_t ticket, double* s, double* a, double* d) {
  if (!ctx) return LSMC_EINVAL;
  std::lock_guard<std::mutex> g(ctx->mu);
  auto it = ctx->tickets.find(ticket);
  if (it == ctx->tickets.end()) {
    auto h = ctx->history.find(ticket);
    if (h == ctx->history.end()) return LSMC_ENOTFOUND;
    if (s) *s = h->second[0];
    if (a) *a = h->second[1];
    if (d) *d = h->second[2];
    return LSMC_OK;
  }
  if (s) *s = it->second->t_submit;
  if (a) *a = it->second->t_admit;
  if (d) *d = it->second->t_done;
  return LSMC_OK;
}

// ---- autotuner ----------------------------------------------------------------
int lsmc_autotune(lsmc_ctx* ctx, const lsmc_request* reqs, size_t n, uint32_t* best_sub,
                  uint32_t* best_ppt, double* best_ms) {
  if (!ctx || !reqs || !n) return LSMC_EINVAL;
  cudaSetDevice(ctx->device);
  PlanOptions o;
  int rc = plan_options(ctx, reqs, n, &o);
  if (rc) return rc;
  const uint64_t key = tune_key(reqs, n, o);
  const uint64_t tiles0 = std::max<uint64_t>(1, 1ull << (key & 0xffffffffu));
  const int dppt = backward_ppt_default(o.precision);
  const uint32_t saved_sub = ctx->sub_override, saved_ppt = ctx->ppt_override;
  uint32_t best = 0;
  double best_t = 1e300;
  // strikes on both sides of S0 in one request: the in-the-money half tiles
  // are worth a trial
  bool mixed_moneyness = false;
  for (size_t i = 0; i < n; ++i) {
    bool itm = false, otm = false;
    for (uint32_t k = 0; k < reqs[i].n_strikes; ++k)
      (itm_at_spot(reqs[i], k) ? itm : otm) = true;
    mixed_moneyness = mixed_moneyness || (itm && otm);
  }
  // each paths-per-lane choice compiled for the precision, and sub-tiles per
  // job in powers of two while the busiest round keeps >= 8 jobs, uniform
  // and (from 2 up) with the in-the-money strikes' jobs halved
  for (int ppt = 2; ppt <= 8 && rc == LSMC_OK; ppt *= 2) {
    if (!backward_ppt_valid(o.precision, ppt)) continue;
    for (uint32_t cand = 1; cand <= kMaxSub && rc == LSMC_OK; cand *= 2) {
      if (cand > 1 && (uint64_t)cand * ppt * 8 > tiles0 * dppt) break;
      for (int half = 0; half < 2 && rc == LSMC_OK; ++half) {
        if (half && (cand < 2 || !mixed_moneyness)) continue;
        ctx->sub_override = cand | (half ? LSMC_SUB_ITM_HALF : 0u);
        ctx->ppt_override = (uint32_t)ppt;
        lsmc_plan* p = nullptr;
        rc = plan_create_on(ctx, reqs, n, ctx->stream, ctx->user_workspace, &p);
        if (rc) break;
        p->timing = true;
        double ms[4] = {0, 0, 0, 0};
        uint32_t launches = 0;
        rc = plan_enqueue(p, true);  // warm-up launch, then the timed one
        if (rc == LSMC_OK) rc = plan_collect(p, nullptr);
        if (rc == LSMC_OK) rc = lsmc_plan_kernel_times(p, ms, &launches);
        if (rc == LSMC_OK) rc = plan_enqueue(p, true);
        if (rc == LSMC_OK) rc = plan_collect(p, nullptr);
        if (rc == LSMC_OK) rc = lsmc_plan_kernel_times(p, ms, &launches);
        plan_free(p);
        if (rc) break;
        if (ms[2] < best_t) { best_t = ms[2]; best = ((uint32_t)ppt << 16) | ctx->sub_override; }
      }
    }
  }
  ctx->sub_override = saved_sub;
  ctx->ppt_override = saved_ppt;
  if (rc && !best) return rc;
  ctx->tuned[key] = best;
  if (best_sub) *best_sub = best & 0xffffu;
  if (best_ppt) *best_ppt = best >> 16;
  if (best_ms) *best_ms = best_t;
  return LSMC_OK;
}

// ---- stage entry points ------------------------------------------------------------
int lsmc_philox(const uint32_t* d_ctr, uint32_t k0, uint32_t k1, uint32_t* d_out, size_t n,
                void* s) {
  if ((!d_ctr || !d_out) && n) return LSMC_EINVAL;
  LSMC_CUDA(launch_philox(d_ctr, k0, k1, d_out, n, (cudaStream_t)s));
  return LSMC_OK;
}

int lsmc_draws(uint64_t seed, uint32_t stream_id, const uint32_t* d_path, const uint32_t* d_step,
               size_t n, int32_t precision, void* d_out, void* s) {
  if ((!d_path || !d_step || !d_out) && n) return LSMC_EINVAL;
  if (precision != LSMC_FP64 && precision != LSMC_MIXED && precision != LSMC_DF)
    return LSMC_EINVAL;
  LSMC_CUDA(launch_draws(seed, stream_id, d_path, d_step, n, precision, d_out,
                         (cudaStream_t)s));
  return LSMC_OK;
}

int lsmc_exp(const void* d_x, void* d_y, size_t n, int32_t precision, void* s) {
  if ((!d_x || !d_y) && n) return LSMC_EINVAL;
  if (precision != LSMC_FP64 && precision != LSMC_MIXED && precision != LSMC_DF)
    return LSMC_EINVAL;
  return cuda_status(launch_exp(d_x, d_y, n, precision, (cudaStream_t)s));
}

int lsmc_quantile(const void* d_u, void* d_z, size_t n, int32_t precision, void* s) {
  if ((!d_u || !d_z) && n) return LSMC_EINVAL;
  if (precision == LSMC_DF) return LSMC_ENOTIMPL;
  if (precision != LSMC_FP64 && precision != LSMC_MIXED) return LSMC_EINVAL;
  return cuda_status(launch_quantile(d_u, d_z, n, precision, (cudaStream_t)s));
}

static int stage_plan(const lsmc_heston* m, double T, int32_t scheme, int32_t precision,
                      uint32_t P, uint32_t N, int32_t basis, const lsmc_contract* c,
                      uint64_t seed, uint32_t stream_id, cudaStream_t s, lsmc_plan** out) {
  lsmc_contract cc{LSMC_PUT, LSMC_AMERICAN, m ? m->S0 : 1.0, T};
  if (c) cc = *c;
  lsmc_request q = default_request(m, &cc, P, N, basis, nullptr, seed);
  q.bumps.greek_mask = 0;
  q.precision = precision;
  q.scheme = scheme;
  q.stream_id = stream_id;
  PlanOptions o;
  int rc = plan_options(nullptr, &q, 1, &o);
  if (rc) return rc;
  o.raw_paths = true;
  std::unique_ptr<lsmc_plan> p(new (std::nothrow) lsmc_plan());
  if (!p) return LSMC_ENOMEM;
  p->stream = s;
  rc = build_layout(&q, 1, o, &p->L);
  if (rc) return rc;
  // paths live in caller memory: drop the path region, rows are P apart
  p->L.total_bytes -= p->L.bytes_paths;
  p->L.bytes_paths = 0;
  for (auto& G : p->L.groups) G.ld = P;
  *out = p.release();
  return LSMC_OK;
}

int lsmc_multi_asset_max(const lsmc_heston* models, uint32_t n_assets, double T, int32_t scheme,
                         int32_t precision, double rho_assets, uint32_t n_paths, uint32_t n_steps,
                         uint64_t seed, uint32_t stream_id, void* d_M, void* s) {
  if (!models || !d_M || n_assets == 0 || n_assets > (uint32_t)kMaxAssets) return LSMC_EINVAL;
  if (n_paths == 0 || n_steps == 0 || n_paths > (1u << 30) || n_steps > (1u << 20))
    return LSMC_EINVAL;
  if (!(rho_assets >= 0.0 && rho_assets <= 1.0)) return LSMC_EINVAL;
  if ((uint64_t)n_paths * (n_steps + 1) >= (1ull << 40)) return LSMC_EINVAL;
  MultiArgs a{};
  for (uint32_t i = 0; i < n_assets; ++i) {
    // the per-asset checks of a pricing request
    const lsmc_contract cc{LSMC_PUT, LSMC_EUROPEAN, 1.0, T};
    const lsmc_request q = default_request(&models[i], &cc, 1, 1, LSMC_BASIS_S2, nullptr, 0);
    const int rc = validate_request(q, precision, scheme);
    if (rc) return rc;
    const lsmc_heston& m = models[i];
    a.assets[i] = MultiModel{m.S0, m.r, m.q, m.v0, m.kappa, m.theta, m.xi, m.rho};
  }
  a.n_assets = n_assets;
  a.P = n_paths;
  a.N = n_steps;
  a.stream_id = stream_id;
  a.seed = seed;
  a.T = T;
  a.sqrt_rho = std::sqrt(rho_assets);
  a.sqrt_1m_rho = std::sqrt(1.0 - rho_assets);
  a.M = d_M;
#ifdef LSMC_CHECKED
  add_range(a.chk, d_M, (size_t)(n_steps + 1) * n_paths * value_bytes(precision));
  if (check_word(&a.chk.err, &a.chk.info) != LSMC_OK) return LSMC_ECUDA;
#endif
  return cuda_status(launch_multi_max(a, precision, scheme, (cudaStream_t)s));
}

int lsmc_paths(const lsmc_heston* m, double T, int32_t scheme, int32_t precision, uint32_t P,
               uint32_t N, uint64_t seed, uint32_t stream_id, void* d_S, void* d_V, void* s) {
  if (!m || !d_S || !d_V) return LSMC_EINVAL;
  lsmc_plan* p = nullptr;
  int rc = stage_plan(m, T, scheme, precision, P, N, LSMC_BASIS_SV2, nullptr, seed, stream_id,
                      (cudaStream_t)s, &p);
  if (rc) return rc;
  rc = plan_alloc(p, false, true);
  if (rc == LSMC_OK) rc = plan_bind_and_upload(p, d_S, d_V, nullptr);
  p->run_backward = p->run_greeks = false;
  if (rc == LSMC_OK) {
    const cudaError_t e = launch_forward(p->fa, precision, scheme, p->stream);
    rc = cuda_status(e);
  }
  plan_free(p);
  return rc;
}

int lsmc_backward(const void* d_S, const void* d_V, uint32_t P, uint32_t N, int32_t precision,
                  const lsmc_heston* m, const lsmc_contract* c, int32_t basis, double* d_out,
                  double* d_beta, uint32_t* d_nsing, void* s) {
  if (!d_S || !m || !c || !d_out) return LSMC_EINVAL;
  if (basis == LSMC_BASIS_SV2 && !d_V) return LSMC_EINVAL;
  const int scheme = m->xi > 0 ? LSMC_SCHEME_QE : LSMC_SCHEME_FT_EULER;
  lsmc_plan* p = nullptr;
  int rc = stage_plan(m, c->T, scheme, precision, P, N, basis, c, 0, 0, (cudaStream_t)s, &p);
  if (rc) return rc;
  p->run_forward = p->run_greeks = false;
  rc = plan_alloc(p, false, true);
  if (rc == LSMC_OK && d_beta)
    rc = cuda_status(cudaMemsetAsync(d_beta, 0xFF, sizeof(double) * 6 * N, p->stream));
  if (rc == LSMC_OK) rc = plan_bind_and_upload(p, const_cast<void*>(d_S), const_cast<void*>(d_V), d_beta);
  if (rc == LSMC_OK) rc = plan_enqueue(p);
  if (rc == LSMC_OK) {
    // price, se, european, continuation, near ties are the first five fields
    rc = cuda_status(cudaMemcpyAsync(d_out, p->d_results, 5 * sizeof(double),
                                     cudaMemcpyDeviceToDevice, p->stream));
    if (rc == LSMC_OK && d_nsing)
      rc = cuda_status(cudaMemcpyAsync(d_nsing, &p->d_results->singular, sizeof(uint32_t),
                                       cudaMemcpyDeviceToDevice, p->stream));
    if (rc == LSMC_OK) {
      Control ctl{};
      rc = cuda_status(cudaMemcpyAsync(&ctl, p->d_ctl, sizeof(Control), cudaMemcpyDeviceToHost, p->stream));
      if (rc == LSMC_OK) rc = cuda_status(cudaStreamSynchronize(p->stream));
      if (rc == LSMC_OK && ctl.error) rc = ctl.error == kDevErrTimeout ? LSMC_ETIMEOUT : LSMC_ECUDA;
    }
  }
  plan_free(p);
  return rc;
}

}  // extern "C"

// ---- backward pass with caller-provided scratch ----------------------------------
namespace lsmc {

int backward_in_scratch(void* scratch, size_t scratch_bytes, const void* d_S, const void* d_V,
                        uint32_t P, uint32_t N, int32_t precision, const lsmc_heston* m,
                        const lsmc_contract* c, int32_t basis, double* d_out, double* d_beta,
                        uint32_t* d_nsing, cudaStream_t s) {
  if (!scratch || !d_S || !m || !c || !d_out) return LSMC_EINVAL;
  if (basis == LSMC_BASIS_SV2 && !d_V) return LSMC_EINVAL;
  const int scheme = m->xi > 0 ? LSMC_SCHEME_QE : LSMC_SCHEME_FT_EULER;
  lsmc_plan* p = nullptr;
  int rc = stage_plan(m, c->T, scheme, precision, P, N, basis, c, 0, 0, s, &p);
  if (rc) return rc;
  std::unique_ptr<lsmc_plan> owner(p);
  if (p->L.total_bytes > scratch_bytes) return LSMC_ENOMEM;
  p->run_forward = p->run_greeks = false;
  p->dev = (char*)scratch;  // borrowed: never freed here
  if (d_beta) rc = cuda_status(cudaMemsetAsync(d_beta, 0xFF, sizeof(double) * 6 * N, s));
  if (rc == LSMC_OK) rc = plan_bind_and_upload(p, const_cast<void*>(d_S), const_cast<void*>(d_V), d_beta);
  if (rc == LSMC_OK) rc = plan_enqueue(p);
  if (rc == LSMC_OK)
    rc = cuda_status(cudaMemcpyAsync(d_out, p->d_results, 5 * sizeof(double),
                                     cudaMemcpyDeviceToDevice, s));
  if (rc == LSMC_OK && d_nsing)
    rc = cuda_status(cudaMemcpyAsync(d_nsing, &p->d_results->singular, sizeof(uint32_t),
                                     cudaMemcpyDeviceToDevice, s));
  Control ctl{};
  if (rc == LSMC_OK)
    rc = cuda_status(cudaMemcpyAsync(&ctl, p->d_ctl, sizeof(Control), cudaMemcpyDeviceToHost, s));
  // whatever was enqueued above reads or writes the shared scratch: wait for
  // it on every path, a failed one included, so the call never returns while
  // its kernels still use the array (the first error is kept)
  const int sync_rc = cuda_status(cudaStreamSynchronize(s));
  if (rc == LSMC_OK) rc = sync_rc;
  if (rc == LSMC_OK && ctl.error) rc = ctl.error == kDevErrTimeout ? LSMC_ETIMEOUT : LSMC_ECUDA;
  p->dev = nullptr;
  return rc;
}

}  // namespace lsmc
