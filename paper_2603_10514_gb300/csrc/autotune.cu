// autotune.cu -- the library's autotuner of the emulated-FP64 products' launch plans.
//
// A plan of the modular product (gemm_oz.cu) is the cap on its column-tile width (256, 192
// or 128 columns per CTA; the tiles are then made as even as possible) and its number of K
// splits (1 or 2).  The best plan depends on the product's shape: how many CTAs the grid
// holds against the 152 SMs, how much of each tile is padding, and whether the per-CTA
// fixed costs are amortised.  Because the modular products are exact integer arithmetic,
// every plan gives bit-identical results, so the tuner times the candidates in place on the
// caller's own data (each candidate overwrites the same output with the same values) the
// first time a shape bucket is met, and keeps the fastest.  Buckets: the rows M and the
// inner dimension K in quarter octaves (round(4 log2)), the columns N in steps of 32.  The
// table is process-wide (the plans are properties of the GPU and the shapes) and guarded
// by a mutex (batch sessions call from several threads).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "../../include/chase_gb300.h"
#include "common.cuh"
#include "kernels.h"

namespace chase {

namespace {

struct Entry {
  OzPlan plan;
  double seconds;
  int shape_M, shape_N, shape_K;  // the shape it was measured on
};

std::mutex& table_mutex() {
  static std::mutex m;
  return m;
}
std::map<std::tuple<int, int, int>, Entry>& table() {
  static std::map<std::tuple<int, int, int>, Entry> t;
  return t;
}

std::tuple<int, int, int> key_of(int M, int N, int kp) {
  return std::make_tuple((int)std::lround(4.0 * std::log2((double)std::max(M, 1))), (N + 31) / 32,
                         (int)std::lround(4.0 * std::log2((double)std::max(kp, 1))));
}

}  // namespace

bool oz_plan_lookup(int M, int N, int kp, OzPlan* plan) {
  std::lock_guard<std::mutex> g(table_mutex());
  auto it = table().find(key_of(M, N, kp));
  if (it == table().end()) return false;
  *plan = it->second.plan;
  return true;
}

void oz_plan_store(int M, int N, int kp, const OzPlan& plan, double seconds) {
  std::lock_guard<std::mutex> g(table_mutex());
  table()[key_of(M, N, kp)] = Entry{plan, seconds, M, N, kp};
}

int oz_plan_candidates(int N, OzPlan* out, int cap) {
  // distinct (tile width, splits) pairs for N columns
  int n = 0;
  int seen_bn[3] = {0, 0, 0};
  const int caps[3] = {256, 192, 128};
  for (int c = 0; c < 3; ++c) {
    const int ntile = (N + caps[c] - 1) / caps[c];
    const int bn = ((N + ntile - 1) / ntile + 15) / 16 * 16;
    bool dup = false;
    for (int d = 0; d < c; ++d) dup |= (seen_bn[d] == bn);
    seen_bn[c] = bn;
    if (dup) continue;
    for (int s = 1; s <= kOzMaxSplits && n < cap; ++s) out[n++] = OzPlan{caps[c], s};
  }
  return n;
}

}  // namespace chase

extern "C" {

int chase_autotune_table(char* buf, size_t cap, size_t* needed) {
  if (cap > 0 && !buf) return -1;
  std::string s;
  {
    std::lock_guard<std::mutex> g(chase::table_mutex());
    char line[256];
    for (const auto& kv : chase::table()) {
      const chase::Entry& e = kv.second;
      snprintf(line, sizeof line,
               "ozm M=%d N=%d K=%d bucket=(%d,%d,%d) tile_cap=%d splits=%d seconds=%.6e\n", e.shape_M,
               e.shape_N, e.shape_K, std::get<0>(kv.first), std::get<1>(kv.first),
               std::get<2>(kv.first), e.plan.bn_max, e.plan.splits, e.seconds);
      s += line;
    }
  }
  if (needed) *needed = s.size() + 1;
  if (cap > 0) {
    const size_t m = std::min(cap - 1, s.size());
    memcpy(buf, s.data(), m);
    buf[m] = '\0';
  }
  return CHASE_OK;
}

int chase_autotune_clear(void) {
  std::lock_guard<std::mutex> g(chase::table_mutex());
  chase::table().clear();
  return CHASE_OK;
}

}  // extern "C"
