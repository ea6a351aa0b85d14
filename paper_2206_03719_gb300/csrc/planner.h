// planner.h -- host planner: request validation, scenario expansion, path
// group folding and the device tables of one launch (internal).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/lsmc.h"
#include "plan.h"

namespace lsmc {

// First-fit sub-allocator over one device range (256-byte granules).
class Arena {
 public:
  void reset(void* base, size_t bytes);
  bool active() const { return base_ != nullptr; }
  void* alloc(size_t bytes);
  void free(void* p);
  size_t capacity() const { return size_; }
  size_t used() const;
  size_t largest_free() const;

 private:
  struct Block { size_t off, size; };
  char* base_ = nullptr;
  size_t size_ = 0;
  std::vector<Block> free_;   // sorted by offset
  std::vector<Block> used_;
  mutable std::mutex mu_;
};

struct Scenario {
  int32_t kind;
  lsmc_heston model;
  double T;
};

// Bump-and-revalue scenarios of a request, in layout order:
// base, S+, S-, S+ (gamma), S- (gamma), v0+, v0-, r+, r-, T-, T+.
int expand_scenarios(const lsmc_request& req, std::vector<Scenario>* out);

// Checks a request; LSMC_OK or LSMC_EINVAL.
int validate_request(const lsmc_request& req, int precision, int scheme);

struct PlanOptions {
  int precision = LSMC_FP64;
  int scheme = LSMC_SCHEME_QE;
  int basis = LSMC_BASIS_S2;
  bool raw_paths = false;       // stage entry point: E rows are S itself
  uint32_t sub = 1;             // sub-tiles per backward job (| LSMC_SUB_ITM_HALF)
  std::vector<uint32_t> sub_req; // per request (if not empty: overrides sub)
  uint32_t ppt = 0;             // paths per thread of a sub-tile (0: the precision's default)
  // regenerate mode: no path store; states saved every ck_stride dates and
  // each segment of ck_stride dates simulated again before its backward rounds
  bool regen = false;
  uint32_t ck_stride = 0;
  bool oos = false;             // out-of-sample pricing pass
  int store = 0;                // element type of the E/V rows (kStore*)
};

// Paths per lane of a plan's backward sub-tiles.
int plan_ppt(const PlanOptions& o);

// Largest number of sub-tiles per backward job.
constexpr uint32_t kMaxSub = 64;

// Whether strike K of request q is in the money at the request's S0 (a put
// struck above it, a call below): with LSMC_SUB_ITM_HALF such strikes of a
// request with several strikes take half the sub-tiles per job.
bool itm_at_spot(const lsmc_request& q, uint32_t k);

// Sub-tiles per backward job so that the busiest round has about
// jobs_per_worker jobs for each of `workers` resident CTAs.
uint32_t choose_sub(const lsmc_request* reqs, size_t n, int precision, int ppt,
                    uint32_t workers, uint32_t jobs_per_worker = 4);

// Sizes and host tables of one launch; device pointers are bound later.
struct PlanLayout {
  PlanOptions opt;
  std::vector<FwdContract> contracts;
  std::vector<FwdGroup> groups;
  std::vector<BwdInstance> inst;          // sorted by gens, descending
  std::vector<unsigned long long> round_off;
  std::vector<uint32_t> cum_tiles, active;
  std::vector<GreekOut> greeks;
  std::vector<uint32_t> req_info;         // per request: instances, first GreekOut, GreekOuts
  // region offsets (bytes) of each group's E and V rows (V: SIZE_MAX if not
  // stored) and of each sorted instance's Y, partials and scale table
  std::vector<size_t> group_E_off, group_V_off;
  // regenerate mode: each group's saved states (x and v at dates k ck_stride)
  std::vector<size_t> group_CX_off, group_CV_off;
  uint32_t n_segments = 0;                // regenerate mode: segments of dates
  // scale: the date tables; beta / oos_partial (out-of-sample mode, inside
  // the same region): coefficients of every date, the pricing pass's sums
  struct InstOff {
    size_t y, partial, scale, beta = SIZE_MAX, oos_partial = SIZE_MAX, oos_tab = SIZE_MAX,
           oos_screen = SIZE_MAX;
    uint32_t group;
  };
  std::vector<InstOff> inst_off;
  uint32_t n_results = 0;                 // BwdResult slots
  uint32_t fwd_blocks = 0;
  uint64_t total_jobs = 0;
  uint64_t generated_path_steps = 0, lsmc_path_steps = 0;
  // device bytes of each region
  size_t bytes_paths = 0, bytes_y = 0, bytes_partial = 0, bytes_scale = 0;
  size_t bytes_tables = 0, bytes_state = 0, bytes_results = 0, bytes_out = 0;
  size_t total_bytes = 0;
};

int build_layout(const lsmc_request* reqs, size_t n, const PlanOptions& opt,
                 PlanLayout* L);

}  // namespace lsmc
