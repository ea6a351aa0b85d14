// planner.cpp -- host planner (validation, scenario table, path-group
// folding, job tables, device layout) and the workspace arena.
#include "planner.h"

#include <algorithm>
#include <cmath>
#include <cstring>

#include "kernels.h"

namespace lsmc {

// ---- arena -------------------------------------------------------------------
static size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

void Arena::reset(void* base, size_t bytes) {
  std::lock_guard<std::mutex> g(mu_);
  base_ = (char*)base;
  size_ = bytes / 256 * 256;
  free_.clear();
  used_.clear();
  if (base_ && size_) free_.push_back({0, size_});
}

void* Arena::alloc(size_t bytes) {
  std::lock_guard<std::mutex> g(mu_);
  if (!base_) return nullptr;
  bytes = round_up(bytes ? bytes : 1, 256);
  for (size_t i = 0; i < free_.size(); ++i) {
    if (free_[i].size >= bytes) {
      Block b{free_[i].off, bytes};
      free_[i].off += bytes;
      free_[i].size -= bytes;
      if (free_[i].size == 0) free_.erase(free_.begin() + i);
      used_.push_back(b);
      return base_ + b.off;
    }
  }
  return nullptr;
}

void Arena::free(void* p) {
  if (!p) return;
  std::lock_guard<std::mutex> g(mu_);
  const size_t off = (size_t)((char*)p - base_);
  for (size_t i = 0; i < used_.size(); ++i) {
    if (used_[i].off != off) continue;
    Block b = used_[i];
    used_.erase(used_.begin() + i);
    auto it = std::lower_bound(free_.begin(), free_.end(), b,
                               [](const Block& x, const Block& y) { return x.off < y.off; });
    it = free_.insert(it, b);
    // coalesce with neighbours
    size_t k = (size_t)(it - free_.begin());
    if (k + 1 < free_.size() && free_[k].off + free_[k].size == free_[k + 1].off) {
      free_[k].size += free_[k + 1].size;
      free_.erase(free_.begin() + k + 1);
    }
    if (k > 0 && free_[k - 1].off + free_[k - 1].size == free_[k].off) {
      free_[k - 1].size += free_[k].size;
      free_.erase(free_.begin() + k);
    }
    return;
  }
}

size_t Arena::used() const {
  std::lock_guard<std::mutex> g(mu_);
  size_t s = 0;
  for (const auto& b : used_) s += b.size;
  return s;
}

size_t Arena::largest_free() const {
  std::lock_guard<std::mutex> g(mu_);
  size_t s = 0;
  for (const auto& b : free_) s = std::max(s, b.size);
  return s;
}

// ---- validation ----------------------------------------------------------------
static bool finite(double x) { return std::isfinite(x); }

int validate_request(const lsmc_request& q, int precision, int scheme) {
  const lsmc_heston& m = q.model;
  const double vals[] = {m.S0, m.r, m.q, m.v0, m.kappa, m.theta, m.xi, m.rho, q.T,
                         q.bumps.rel_dS, q.bumps.rel_dS_gamma, q.bumps.rel_dv0,
                         q.bumps.abs_dr, q.bumps.abs_dT};
  for (double v : vals)
    if (!finite(v)) return LSMC_EINVAL;
  if (!(m.S0 > 0) || !(q.T > 0) || m.v0 < 0 || !(m.kappa > 0) || !(m.theta > 0) ||
      m.xi < 0 || std::fabs(m.rho) > 1.0)
    return LSMC_EINVAL;
  if (scheme != LSMC_SCHEME_QE && scheme != LSMC_SCHEME_FT_EULER) return LSMC_EINVAL;
  if (scheme == LSMC_SCHEME_QE && !(m.xi > 0)) return LSMC_EINVAL;
  if (precision != LSMC_FP64 && precision != LSMC_MIXED && precision != LSMC_DF) return LSMC_EINVAL;
  if (q.type != LSMC_PUT && q.type != LSMC_CALL) return LSMC_EINVAL;
  if (q.style != LSMC_AMERICAN && q.style != LSMC_EUROPEAN) return LSMC_EINVAL;
  if (q.basis != LSMC_BASIS_S2 && q.basis != LSMC_BASIS_SV2) return LSMC_EINVAL;
  if (q.flags & ~(uint32_t)(LSMC_FLAG_REGENERATE | LSMC_FLAG_OUT_OF_SAMPLE |
                            LSMC_FLAG_STORE_FP16 | LSMC_FLAG_STORE_BF16))
    return LSMC_EINVAL;
  if ((q.flags & LSMC_FLAG_STORE_FP16) && (q.flags & LSMC_FLAG_STORE_BF16)) return LSMC_EINVAL;
  if (q.n_paths == 0 || q.n_steps == 0 || q.n_strikes == 0 || !q.strikes) return LSMC_EINVAL;
  if (q.n_paths > (1u << 30) || q.n_steps > (1u << 20) || q.n_strikes > 4096) return LSMC_EINVAL;
  for (uint32_t k = 0; k < q.n_strikes; ++k)
    if (!finite(q.strikes[k]) || !(q.strikes[k] > 0)) return LSMC_EINVAL;
  std::vector<Scenario> sc;
  return expand_scenarios(q, &sc) < 0 ? LSMC_EINVAL : LSMC_OK;
}

int expand_scenarios(const lsmc_request& q, std::vector<Scenario>* out) {
  const lsmc_bumps& b = q.bumps;
  const uint32_t mask = b.greek_mask;
  if (mask & ~31u) return LSMC_EINVAL;
  out->clear();
  auto add = [&](int kind, lsmc_heston m, double T) { out->push_back({kind, m, T}); };
  const lsmc_heston& m0 = q.model;
  add(kScBase, m0, q.T);
  const bool want_delta = mask & LSMC_GREEK_DELTA, want_gamma = mask & LSMC_GREEK_GAMMA;
  const bool gamma_shares = b.rel_dS_gamma == 0.0 || b.rel_dS_gamma == b.rel_dS;
  if (want_delta || (want_gamma && gamma_shares)) {
    if (!(b.rel_dS > 0 && b.rel_dS < 1)) return LSMC_EINVAL;
    lsmc_heston up = m0, dn = m0;
    up.S0 = m0.S0 * (1.0 + b.rel_dS);
    dn.S0 = m0.S0 * (1.0 - b.rel_dS);
    add(kScSUp, up, q.T);
    add(kScSDn, dn, q.T);
  }
  if (want_gamma && !gamma_shares) {
    if (!(b.rel_dS_gamma > 0 && b.rel_dS_gamma < 1)) return LSMC_EINVAL;
    lsmc_heston up = m0, dn = m0;
    up.S0 = m0.S0 * (1.0 + b.rel_dS_gamma);
    dn.S0 = m0.S0 * (1.0 - b.rel_dS_gamma);
    add(kScSgUp, up, q.T);
    add(kScSgDn, dn, q.T);
  }
  if (mask & LSMC_GREEK_VEGA) {
    if (!(b.rel_dv0 > 0 && b.rel_dv0 < 1) || !(m0.v0 > 0)) return LSMC_EINVAL;
    lsmc_heston up = m0, dn = m0;
    up.v0 = m0.v0 * (1.0 + b.rel_dv0);
    dn.v0 = m0.v0 * (1.0 - b.rel_dv0);
    add(kScVUp, up, q.T);
    add(kScVDn, dn, q.T);
  }
  if (mask & LSMC_GREEK_RHO) {
    if (!(b.abs_dr > 0)) return LSMC_EINVAL;
    lsmc_heston up = m0, dn = m0;
    up.r = m0.r + b.abs_dr;
    dn.r = m0.r - b.abs_dr;
    add(kScRUp, up, q.T);
    add(kScRDn, dn, q.T);
  }
  if (mask & LSMC_GREEK_THETA) {
    if (!(b.abs_dT > 0 && b.abs_dT < q.T)) return LSMC_EINVAL;
    add(kScTDn, m0, q.T - b.abs_dT);
    add(kScTUp, m0, q.T + b.abs_dT);
  }
  return (int)out->size();
}

// Scenarios whose paths are one simulation: same T and same model except S0
// (x = ln(S/S0) does not depend on S0) and r (the variance path does not
// depend on r, and x moves by n (dr) dt).
static bool same_path_group(const Scenario& a, const lsmc_heston& g, double gT) {
  const lsmc_heston& m = a.model;
  return a.T == gT && m.v0 == g.v0 && m.kappa == g.kappa && m.theta == g.theta &&
         m.xi == g.xi && m.rho == g.rho && m.q == g.q;
}

int plan_ppt(const PlanOptions& o) {
  return o.ppt && backward_ppt_valid(o.precision, (int)o.ppt) ? (int)o.ppt
                                                             : backward_ppt_default(o.precision);
}

bool itm_at_spot(const lsmc_request& q, uint32_t k) {
  return q.type == LSMC_PUT ? q.strikes[k] > q.model.S0 : q.strikes[k] < q.model.S0;
}

uint32_t choose_sub(const lsmc_request* reqs, size_t n, int precision, int ppt,
                    uint32_t workers, uint32_t jobs_per_worker) {
  const uint64_t tile0 = (uint64_t)backward_tile(precision, ppt);
  uint64_t tiles = 0;  // sub-tiles of the first round, over all instances
  for (size_t i = 0; i < n; ++i) {
    std::vector<Scenario> sc;
    if (expand_scenarios(reqs[i], &sc) < 0) continue;
    tiles += (uint64_t)sc.size() * reqs[i].n_strikes * ((reqs[i].n_paths + tile0 - 1) / tile0);
  }
  const uint64_t want = (uint64_t)std::max<uint32_t>(1, workers) * std::max<uint32_t>(1, jobs_per_worker);
  const uint64_t sub = tiles / want;
  return (uint32_t)std::min<uint64_t>(kMaxSub, std::max<uint64_t>(1, sub));
}

int build_layout(const lsmc_request* reqs, size_t n, const PlanOptions& opt,
                 PlanLayout* L) {
  *L = PlanLayout();
  L->opt = opt;
  const size_t real = value_bytes(opt.precision);
  const size_t rowb = row_bytes(opt.precision, opt.store);  // an element of the E/V rows
  const uint32_t tile0 = (uint32_t)backward_tile(opt.precision, plan_ppt(opt));
  const bool store_v = opt.basis == LSMC_BASIS_SV2;
  // device offsets are relative to the region starts; the caller binds them
  size_t off_paths = 0, off_y = 0, off_partial = 0, off_scale = 0;
  std::vector<BwdInstance> inst;
  std::vector<PlanLayout::InstOff> offs;
  for (size_t ci = 0; ci < n; ++ci) {
    const lsmc_request& q = reqs[ci];
    std::vector<Scenario> sc;
    if (expand_scenarios(q, &sc) < 0) return LSMC_EINVAL;
    const uint32_t P = q.n_paths, N = q.n_steps;
    const uint64_t ld = round_up(P, 32);
    // fold scenarios onto path groups
    std::vector<int> sc_group(sc.size());
    std::vector<double> gT;       // maturity of each group of this contract
    const uint32_t group0 = (uint32_t)L->groups.size();
    for (size_t s = 0; s < sc.size(); ++s) {
      int found = -1;
      for (size_t g = 0; g < gT.size(); ++g) {
        const FwdGroup& G = L->groups[group0 + g];
        lsmc_heston gm{0, G.r, G.q, G.v0, G.kappa, G.theta, G.xi, G.rho};
        if (same_path_group(sc[s], gm, gT[g])) { found = (int)g; break; }
      }
      if (found < 0) {
        if (gT.size() >= (size_t)kMaxGroups) return LSMC_ENOTIMPL;
        FwdGroup G{};
        const lsmc_heston& m = sc[s].model;
        G.v0 = m.v0; G.kappa = m.kappa; G.theta = m.theta; G.xi = m.xi;
        G.rho = m.rho; G.r = m.r; G.q = m.q;
        G.dt = sc[s].T / (double)N;
        G.out_scale = opt.raw_paths ? m.S0 : 1.0;
        G.ld = ld;
        G.E = G.V = G.E_row0 = G.V_row0 = G.CX = G.CV = nullptr;
        // rows of the store: dates 1..N, or in regenerate mode one segment
        // of dates c..c + ck_stride (ck_stride + 1 rows)
        const size_t rows = opt.regen ? (size_t)opt.ck_stride + 1 : (size_t)N;
        L->group_E_off.push_back(off_paths);
        off_paths += round_up(rows * ld * rowb, 256);
        if (store_v) {
          L->group_V_off.push_back(off_paths);
          off_paths += round_up(rows * ld * rowb, 256);
        } else {
          L->group_V_off.push_back(SIZE_MAX);
        }
        if (opt.regen) {
          // saved states x, v at dates k ck_stride, k = 0..n_segments-1
          const size_t segs = (N + opt.ck_stride - 1) / opt.ck_stride;
          L->group_CX_off.push_back(off_paths);
          off_paths += round_up(segs * ld * real, 256);
          L->group_CV_off.push_back(off_paths);
          off_paths += round_up(segs * ld * real, 256);
        } else {
          L->group_CX_off.push_back(SIZE_MAX);
          L->group_CV_off.push_back(SIZE_MAX);
        }
        found = (int)gT.size();
        gT.push_back(sc[s].T);
        L->groups.push_back(G);
      }
      sc_group[s] = found;
    }
    FwdContract C{};
    C.seed = q.seed;
    C.stream_id = q.stream_id;
    C.P = P;
    C.N = N;
    C.group0 = group0;
    C.n_groups = (uint32_t)gT.size();
    C.block0 = L->fwd_blocks;
    L->fwd_blocks += (P + kFwdBlock - 1) / kFwdBlock;
    L->contracts.push_back(C);
    L->generated_path_steps += (uint64_t)P * N * sc.size();
    L->lsmc_path_steps += (uint64_t)P * N * sc.size() * q.n_strikes;

    const uint32_t sub_flags = ci < opt.sub_req.size() ? opt.sub_req[ci] : opt.sub;
    const bool itm_half = (sub_flags & LSMC_SUB_ITM_HALF) != 0 && q.n_strikes > 1;
    const uint32_t sub = std::max<uint32_t>(1, sub_flags & ~LSMC_SUB_ITM_HALF);
    // sub-tiles per job and tiles of strike k
    auto sub_of = [&](uint32_t k) {
      return itm_half && itm_at_spot(q, k) ? std::max<uint32_t>(1, sub / 2) : sub;
    };
    auto tiles_of = [&](uint32_t k) { return (P + tile0 * sub_of(k) - 1) / (tile0 * sub_of(k)); };
    for (uint32_t k = 0; k < q.n_strikes; ++k)
      if ((uint64_t)tiles_of(k) * N >= (1ull << 31)) return LSMC_EINVAL;
    std::vector<GreekOut> gos(q.n_strikes);
    for (auto& g : gos) {
      for (int k = 0; k < kScCount; ++k) g.res[k] = -1;
      g.mask = q.bumps.greek_mask;
      g.S0 = q.model.S0; g.v0 = q.model.v0;
      g.hS = q.bumps.rel_dS; g.hG = q.bumps.rel_dS_gamma; g.hV = q.bumps.rel_dv0;
      g.dR = q.bumps.abs_dr; g.dT = q.bumps.abs_dT;
    }
    for (size_t s = 0; s < sc.size(); ++s) {
      const uint32_t gi = group0 + (uint32_t)sc_group[s];
      const FwdGroup& G = L->groups[gi];
      for (uint32_t k = 0; k < q.n_strikes; ++k) {
        BwdInstance I{};
        I.E = I.V = nullptr;
        I.ld = ld;
        PlanLayout::InstOff o;
        o.group = gi;
        o.y = off_y;
        off_y += round_up((size_t)P * real, 256);
        o.partial = off_partial;
        off_partial += round_up((size_t)tiles_of(k) * kNSum * 8, 256);
        o.scale = off_scale;
        off_scale += round_up((size_t)2 * (N + 1) * 8, 256);
        o.beta = SIZE_MAX;
        if (opt.oos) {  // coefficients of every date, and the pricing pass's tile sums
          o.beta = off_scale;
          off_scale += round_up((size_t)N * 8 * 8, 256);
          o.oos_partial = off_scale;
          off_scale += round_up((size_t)((P + kOosTile - 1) / kOosTile) * 4 * 8, 256);
          o.oos_tab = off_scale;  // the per-date constants in the working precision
          off_scale += round_up((size_t)(N + 1) * kOosConsts * real, 256);
          o.oos_screen = off_scale;  // and the per-date float screens of the test
          off_scale += round_up((size_t)(N + 1) * kScreenBytes, 256);
        }
        I.Y = nullptr;
        I.partial = nullptr;
        I.scale_tab = nullptr;
        I.beta_hist = nullptr;
        I.spot = sc[s].model.S0;
        I.scale0 = opt.raw_paths ? 1.0 : sc[s].model.S0;
        I.dr_dt = (sc[s].model.r - G.r) * G.dt;
        I.r = sc[s].model.r;
        I.dt = G.dt;
        I.T = sc[s].T;
        I.K = q.strikes[k];
        I.theta = sc[s].model.theta;
        I.P = P;
        I.N = N;
        I.tiles = tiles_of(k);
        I.sub = sub_of(k);
        I.gens = q.style == LSMC_EUROPEAN ? 1 : N;
        I.type = q.type;
        I.style = q.style;
        I.basis = opt.basis;
        I.out_index = L->n_results++;
        I.req = (uint32_t)ci;
        gos[k].res[sc[s].kind] = (int32_t)I.out_index;
        inst.push_back(I);
        offs.push_back(o);
      }
    }
    // per request: its instances, first GreekOut and GreekOuts
    L->req_info.push_back((uint32_t)(sc.size() * q.n_strikes));
    L->req_info.push_back((uint32_t)L->greeks.size());
    L->req_info.push_back(q.n_strikes);
    for (auto& g : gos) L->greeks.push_back(g);
  }
  // jobs: round-major over instances sorted by generations (stable)
  std::vector<uint32_t> order(inst.size());
  for (uint32_t i = 0; i < order.size(); ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) {
    return inst[a].gens > inst[b].gens;
  });
  for (uint32_t i : order) {
    L->inst.push_back(inst[i]);
    L->inst_off.push_back(offs[i]);
  }
  inst = L->inst;
  const uint32_t n_inst = (uint32_t)inst.size();
  L->cum_tiles.assign(n_inst + 1, 0);
  for (uint32_t i = 0; i < n_inst; ++i) L->cum_tiles[i + 1] = L->cum_tiles[i] + inst[i].tiles;
  const uint32_t R = n_inst ? inst[0].gens : 0;
  L->round_off.assign(R + 1, 0);
  L->active.assign(R, 0);
  uint32_t act = n_inst;
  for (uint32_t r = 0; r < R; ++r) {
    while (act > 0 && inst[act - 1].gens <= r) --act;
    L->active[r] = act;
    L->round_off[r + 1] = L->round_off[r] + L->cum_tiles[act];
  }
  L->total_jobs = L->round_off[R];

  L->bytes_paths = off_paths;
  if (opt.regen && n > 0)
    L->n_segments = (reqs[0].n_steps + opt.ck_stride - 1) / opt.ck_stride;
  L->bytes_y = off_y;
  L->bytes_partial = off_partial;
  L->bytes_scale = off_scale;
  L->bytes_tables = round_up(sizeof(FwdContract) * L->contracts.size(), 256) +
                    round_up(sizeof(FwdGroup) * L->groups.size(), 256) +
                    round_up(sizeof(BwdInstance) * L->inst.size(), 256) +
                    round_up(sizeof(unsigned long long) * L->round_off.size(), 256) +
                    round_up(sizeof(uint32_t) * L->cum_tiles.size(), 256) +
                    round_up(sizeof(uint32_t) * std::max<size_t>(1, L->active.size()), 256) +
                    round_up(sizeof(GreekOut) * L->greeks.size(), 256) +
                    round_up(sizeof(uint32_t) * L->req_info.size(), 256);
  // state: the instances' states, the control word, the requests' counters
  L->bytes_state = round_up(sizeof(BwdState) * n_inst + sizeof(Control) +
                            sizeof(uint32_t) * n, 256);
  L->bytes_results = round_up(sizeof(BwdResult) * L->n_results, 256);
  L->bytes_out = round_up(sizeof(DevResult) * L->greeks.size(), 256);
  L->total_bytes = L->bytes_tables + L->bytes_state + L->bytes_results + L->bytes_out +
                   L->bytes_scale + L->bytes_partial + L->bytes_y + L->bytes_paths;
  return LSMC_OK;
}

}  // namespace lsmc
