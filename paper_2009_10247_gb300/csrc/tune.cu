// tune.cu -- the schedule autotuner (lp_autotune in include/lp.h).
//
// It runs the handle's own solves under each candidate schedule, times them with CUDA events
// on the caller's stream, checks that every candidate returns the same bits as the first one
// (schedules change the mapping onto the GPU, never the result), and keeps the fastest.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "kernels.h"
#include "program.h"

namespace lp {
namespace {

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  Timer() {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
  }
  ~Timer() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

// One candidate: warm-up, reps timed runs (median), result copied to `bits` for comparison.
// run() issues the solve on the stream; returns LP_OK or an error (candidate skipped on OOM).
template <typename Run>
lp_status time_candidate(Run run, int reps, cudaStream_t s, const void* result, size_t result_bytes,
                         std::vector<uint8_t>& bits, float* ms_out) {
  Timer t;
  lp_status st = run();
  if (st != LP_OK) return st;
  std::vector<float> ts;
  for (int r = 0; r < reps; r++) {
    LP_CUDA(cudaEventRecord(t.a, s));
    if ((st = run()) != LP_OK) return st;
    LP_CUDA(cudaEventRecord(t.b, s));
    LP_CUDA(cudaEventSynchronize(t.b));
    float ms = 0.f;
    LP_CUDA(cudaEventElapsedTime(&ms, t.a, t.b));
    ts.push_back(ms);
  }
  std::sort(ts.begin(), ts.end());
  *ms_out = ts[ts.size() / 2];
  bits.resize(result_bytes);
  LP_CUDA(cudaMemcpyAsync(bits.data(), result, result_bytes, cudaMemcpyDeviceToHost, s));
  LP_CUDA(cudaStreamSynchronize(s));
  return LP_OK;
}

}  // namespace
}  // namespace lp

using namespace lp;

extern "C" lp_status lp_autotune(lp_program* p, uint32_t what, int32_t reps, lp_tune_record* records,
                                 int32_t max_records, int32_t* n_records, void* cuda_stream) {
  NvtxRange nvtx("lp_autotune");
  if (!p) return fail(LP_ERR_INVALID, "program must not be NULL");
  if (p->host_only) return fail(LP_ERR_INVALID, "program was compiled with LP_COMPILE_HOST_ONLY");
  if (what == 0 || (what & ~(LP_TUNE_LEAST | LP_TUNE_STABLE))) return fail(LP_ERR_INVALID, "unknown tune flags");
  if (reps < 1) return fail(LP_ERR_INVALID, "reps must be >= 1");
  if (max_records < 0 || (max_records > 0 && !records)) return fail(LP_ERR_INVALID, "bad records buffer");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const HostMatrix& hm = p->hm;
  const lp_schedule base = p->sched;
  lp_schedule best_least = base, best_stable = base;
  std::vector<lp_tune_record> recs;
  lp_status st = LP_OK;

  if (what & LP_TUNE_LEAST) {
    const size_t out_bytes = (size_t)((hm.n + 63) / 64) * 8;
    if ((st = ensure(p, p->tune_out, std::max<size_t>(out_bytes, 8))) != LP_OK) return st;
    uint64_t* out = (uint64_t*)p->tune_out.p;
    const int occ0 = fixpoint_blocks_per_sm(1, 1, 0), occ1 = fixpoint_stream_blocks_per_sm();
    auto least = [&](int kernel, int blocks, int split, int batch, int map) {
      lp_schedule c = base;  // stable fields stay as they are
      c.fixpoint_kernel = kernel;
      c.fixpoint_blocks_per_sm = blocks;
      c.fixpoint_row_split = split;
      c.fixpoint_chunk_batch = batch;
      c.fixpoint_row_map = map;
      c.fixpoint_stage = 0;
      return c;
    };
    std::vector<lp_schedule> cands;
    for (int b : {0, 4, 2})
      if (b == 0 || b < occ0) cands.push_back(least(0, b, 1, 1, 0));
    for (int G : {2, 4, 8}) cands.push_back(least(0, 0, G, 1, 0));
    for (int G : {1, 2, 4, 8}) cands.push_back(least(0, 0, G, 4, 0));
    for (int m : {1, 2, 3}) cands.push_back(least(0, 0, 1, 1, m));
    for (int b : {0, 1})
      if (occ1 > 0 && (b == 0 || b < occ1)) cands.push_back(least(1, b, 1, 1, 0));
    bool fits3 = false;
    if ((st = block_kernel_fits(p, s, &fits3)) != LP_OK) return st;
    if (fits3) cands.push_back(least(3, 0, 1, 1, 0));
    if (sliced_supported(p))
      for (int stage : {0, 1}) {
        lp_schedule c = least(2, 0, 1, 1, 0);
        c.fixpoint_stage = stage;
        cands.push_back(c);
      }
    std::vector<uint8_t> ref, bits;
    float best = -1.f;
    for (const lp_schedule& c : cands) {
      p->sched = c;
      float ms = -1.f;
      st = time_candidate(
          [&] { return lp_least_model(p, nullptr, out, 1 << 30, 0u, nullptr, cuda_stream); }, reps, s, out,
          out_bytes, bits, &ms);
      if (st == LP_ERR_OOM) {
        recs.push_back({c, (int32_t)LP_TUNE_LEAST, -1.f});
        continue;
      }
      if (st != LP_OK) {
        p->sched = base;
        return st;
      }
      if (ref.empty()) ref = bits;
      else if (bits != ref) {
        p->sched = base;
        return fail(LP_ERR_CUDA, "autotune: least-model schedules disagree");
      }
      recs.push_back({c, (int32_t)LP_TUNE_LEAST, ms});
      if (best < 0.f || ms < best) {
        best = ms;
        best_least = c;
      }
    }
  }

  if (what & LP_TUNE_STABLE) {
    const bool all = hm.k <= 16;
    const int64_t n_guesses = all ? (int64_t(1) << hm.k) : (int64_t(1) << 16);
    const int64_t n_gwords = (n_guesses + 63) / 64;
    const uint64_t* guesses = nullptr;
    if (!all) {  // the first 2^16 guesses, in order
      if ((st = ensure(p, p->tune_in, (size_t)n_guesses * 8)) != LP_OK) return st;
      std::vector<uint64_t> g((size_t)n_guesses);
      std::iota(g.begin(), g.end(), uint64_t(0));
      LP_CUDA(cudaMemcpyAsync(p->tune_in.p, g.data(), g.size() * 8, cudaMemcpyHostToDevice, s));
      LP_CUDA(cudaStreamSynchronize(s));
      guesses = (const uint64_t*)p->tune_in.p;
    }
    if ((st = ensure(p, p->tune_out, (size_t)n_gwords * 8)) != LP_OK) return st;
    uint64_t* mask = (uint64_t*)p->tune_out.p;
    const int occ = stable_blocks_per_sm(false);
    auto stable = [&](int W, int blocks, int split, int frontier) {
      lp_schedule c = best_least;  // least-model fields as chosen above
      c.stable_tile_words = W;
      c.stable_blocks_per_sm = blocks;
      c.stable_row_split = split;
      c.stable_frontier = frontier;
      return c;
    };
    std::vector<lp_schedule> cands;
    for (int W = 1; W <= 32; W *= 2) {
      if (W > 1 && W / 2 >= n_gwords) break;  // wider tiles than the guesses only repeat
      for (int b : {0, occ / 2})
        if (b == 0 || (b > 0 && b < occ)) cands.push_back(stable(W, b, 0, 0));
      if (W < 32) cands.push_back(stable(W, 0, 1, 0));  // with 32-word tiles the row split is the same mapping
      if (W >= 8 || W >= n_gwords) {
        cands.push_back(stable(W, 0, 0, 1));
        cands.push_back(stable(W, 0, 0, 2));
      }
    }
    std::vector<uint8_t> ref, bits;
    float best = -1.f;
    for (const lp_schedule& c : cands) {
      p->sched = c;
      float ms = -1.f;
      st = time_candidate(
          [&] { return lp_stable_models(p, guesses, n_guesses, mask, nullptr, 0, nullptr, 1 << 30, cuda_stream); },
          reps, s, mask, (size_t)n_gwords * 8, bits, &ms);
      if (st == LP_ERR_OOM) {
        recs.push_back({c, (int32_t)LP_TUNE_STABLE, -1.f});
        continue;
      }
      if (st != LP_OK) {
        p->sched = base;
        return st;
      }
      if (ref.empty()) ref = bits;
      else if (bits != ref) {
        p->sched = base;
        return fail(LP_ERR_CUDA, "autotune: stable-model schedules disagree");
      }
      recs.push_back({c, (int32_t)LP_TUNE_STABLE, ms});
      if (best < 0.f || ms < best) {
        best = ms;
        best_stable = c;
      }
    }
  }

  lp_schedule chosen = base;
  if (what & LP_TUNE_LEAST) {
    chosen.fixpoint_kernel = best_least.fixpoint_kernel;
    chosen.fixpoint_blocks_per_sm = best_least.fixpoint_blocks_per_sm;
    chosen.fixpoint_row_split = best_least.fixpoint_row_split;
    chosen.fixpoint_chunk_batch = best_least.fixpoint_chunk_batch;
    chosen.fixpoint_row_map = best_least.fixpoint_row_map;
    chosen.fixpoint_stage = best_least.fixpoint_stage;
  }
  if (what & LP_TUNE_STABLE) {
    chosen.stable_tile_words = best_stable.stable_tile_words;
    chosen.stable_blocks_per_sm = best_stable.stable_blocks_per_sm;
    chosen.stable_row_split = best_stable.stable_row_split;
    chosen.stable_frontier = best_stable.stable_frontier;
  }
  p->sched = chosen;
  for (int32_t i = 0; i < max_records && i < (int32_t)recs.size(); i++) records[i] = recs[i];
  if (n_records) *n_records = (int32_t)recs.size();
  return LP_OK;
}
