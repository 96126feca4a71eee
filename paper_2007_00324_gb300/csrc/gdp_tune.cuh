// Autotuner of the refinement's launch parameters (Rule 2 of the paper:
// trade speculative waste against occupancy).  Included at the end of gdp.cu.
//
// For a sample of PSLGs it builds the CDT once per trial (not timed), runs the
// refinement with every pair (threads per block of the per-candidate kernels,
// per-mesh candidate cap) of the grid below, and keeps the pair with the most
// Steiner points inserted per second of refinement device time.  Each trial
// starts from a fresh CDT of the same inputs, so they all do the same work up
// to the insertion order the cap changes.
#pragma once

namespace {
constexpr int TUNE_BLOCKS[] = {32, 64, 128, 256};
constexpr int TUNE_CAPS[] = {0, 16384, 4096, 1024, 256};
constexpr int TUNE_N = (int)(sizeof(TUNE_BLOCKS) / sizeof(int)) * (int)(sizeof(TUNE_CAPS) / sizeof(int));
}  // namespace

extern "C" {

int gdp_autotune(const double* xy, const int64_t* pt_off, const int32_t* seg, const int64_t* seg_off,
                 int32_t n_meshes, const double* B, const gdp_refine_opts* base, void* stream,
                 gdp_refine_opts* best, double* trials, int32_t trials_cap) {
  if (!xy || !pt_off || !seg_off || n_meshes <= 0 || !best) return GDP_ERR_INPUT;
  std::vector<long long> po(n_meshes + 1), so(n_meshes + 1);
  for (int m = 0; m <= n_meshes; ++m) {
    po[m] = pt_off[m];
    so[m] = seg_off[m];
    if (m && (po[m] - po[m - 1] < 3 || so[m] < so[m - 1])) return GDP_ERR_INPUT;
  }
  if (po[0] != 0 || so[0] != 0 || (so[n_meshes] > 0 && !seg)) return GDP_ERR_INPUT;
  gdp_refine_opts o{};
  if (base) o = *base;
  o.flags = 0;
  double best_rate = -1.0;
  int k = 0;
  for (int b : TUNE_BLOCKS) {
    for (int c : TUNE_CAPS) {
      PoolHost h;
      int st = h.setup(xy, po.data(), seg, so.data(), n_meshes, false, stream);
      if (st == GDP_OK) st = h.build_cdt();
      if (st != GDP_OK) return st;
      o.cand_block = b;
      o.cand_cap = c;
      st = h.refine(B, &o);
      if (st != GDP_OK) return st;
      const double rate = h.stats.refine_ms > 0 ? h.stats.n_steiner / (h.stats.refine_ms * 1e-3) : 0.0;
      if (trials && k < trials_cap) {
        trials[4 * k] = b;
        trials[4 * k + 1] = c;
        trials[4 * k + 2] = h.stats.refine_ms;
        trials[4 * k + 3] = (double)h.stats.n_steiner;
      }
      ++k;
      if (rate > best_rate) {
        best_rate = rate;
        *best = o;
      }
    }
  }
  return GDP_OK;
}

}  // extern "C"
