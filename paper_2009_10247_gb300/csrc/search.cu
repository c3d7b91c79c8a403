// search.cu -- fixed-budget guess sampling with local search over the guessed atoms
// (lp_stable_search in include/lp.h).
//
// Algorithm 2 enumerates all 2^k columns of M_0 (Def. 8); the paper leaves larger k to future
// work (Sec. 5). Here a population of P <= 2048 guesses (one column tile) runs to its fixpoint
// through lp_stable_models, and Algorithm 3 marks the stable columns. For every column the
// fixpoint also implies a guess: bit j = 1 iff the j-th guessed atom q_j is false in it (the
// barred atom q_j-bar should hold). Algorithm 3 accepts a column exactly when the implied guess
// equals the column's own guess. A column that fails moves to its implied guess (a
// Gelfond-Lifschitz step on the guessed atoms). When that returns to the guess it held one round
// earlier (a 2-cycle), only the bits the step would flip are drawn at random, a WalkSAT-like
// move. After a success the column restarts from a fresh random guess. The random bits come from
// a counter-based generator (SplitMix64 of seed, round and column), so a run is reproducible.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "device.cuh"
#include "kernels.h"
#include "program.h"

namespace lp {

// SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number generators", 2014).
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__device__ __forceinline__ uint64_t random_guess(uint64_t seed, int round, int col, uint64_t kmask) {
  return splitmix64(splitmix64(seed ^ ((uint64_t)round << 32)) + (uint64_t)col) & kmask;
}

// Population of the first search round.
__global__ void search_init_kernel(uint64_t* guess, uint64_t* prev, int P, uint64_t seed, uint64_t kmask) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < P; c += gridDim.x * blockDim.x) {
    guess[c] = random_guess(seed, 0, c, kmask);
    prev[c] = ~0ull;  // no previous guess
  }
}

// One update after a round: implied guesses from the fixpoint (tile buffer X, W words per row,
// column c = bit c&63 of word c>>6), stable columns appended to `found`, next population.
__global__ void search_update_kernel(const uint64_t* __restrict__ X, int log2W, const int32_t* __restrict__ q_row,
                                     int k, const uint64_t* __restrict__ stable_mask, uint64_t* guess,
                                     uint64_t* prev, int P, uint64_t seed, int round, uint64_t kmask,
                                     uint64_t* found, unsigned long long* n_found, long long cap) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < P; c += gridDim.x * blockDim.x) {
    const int w = c >> 6, b = c & 63;
    const uint64_t g = guess[c];
    const bool stable = (stable_mask[w] >> b) & 1ull;
    uint64_t next;
    if (stable) {
      const unsigned long long slot = atomicAdd(n_found, 1ull);
      if ((long long)slot < cap) found[slot] = g;
      next = random_guess(seed, round + 1, c, kmask);
    } else {
      uint64_t implied = 0;
      for (int j = 0; j < k; j++) {
        const uint64_t qw = X[((long long)__ldg(q_row + j) << log2W) + w];
        implied |= (uint64_t)(((qw >> b) & 1ull) ^ 1ull) << j;
      }
      if (implied == prev[c]) {  // 2-cycle: redraw only the bits the step would flip
        const uint64_t d = implied ^ g;
        next = (implied & ~d) | (random_guess(seed, round + 1, c, kmask) & d);
      } else {
        next = implied;
      }
    }
    prev[c] = g;
    guess[c] = next;
  }
}

}  // namespace lp

using namespace lp;

extern "C" lp_status lp_stable_search(lp_program* p, int32_t population, int32_t rounds, uint64_t seed,
                                      uint64_t* found, int64_t max_found, int64_t* n_found, void* cuda_stream) {
  NvtxRange nvtx("lp_stable_search");
  if (!p) return fail(LP_ERR_INVALID, "program must not be NULL");
  if (p->host_only) return fail(LP_ERR_INVALID, "program was compiled with LP_COMPILE_HOST_ONLY");
  if (population < 1 || population > 2048) return fail(LP_ERR_INVALID, "population must be in [1, 2048]");
  if (rounds < 1) return fail(LP_ERR_INVALID, "rounds must be >= 1");
  if (max_found < 0 || (max_found > 0 && !found)) return fail(LP_ERR_INVALID, "bad found buffer");
  if (!n_found) return fail(LP_ERR_INVALID, "n_found must not be NULL");
  const HostMatrix& hm = p->hm;
  if (hm.k > 64) return fail(LP_ERR_TOO_MANY_GUESSES, "k > 64 guessed atoms do not fit a guess word");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  lp_status st;
  const int k = hm.k;
  const uint64_t kmask = k >= 64 ? ~0ull : ((1ull << k) - 1ull);
  const int P = population;
  const int n_gwords = (P + 63) / 64;
  int W = 1;
  while (W < n_gwords) W <<= 1;  // one tile holds the whole population

  // internal row of q_j for every guessed atom j (bit order of the guesses)
  std::vector<int32_t> qrow(std::max(k, 1), 0);
  for (int j = 0; j < k; j++)
    for (size_t i = 0; i < hm.bar_row.size(); i++)
      if (hm.bar_row[i] == hm.guess_row[j]) qrow[j] = hm.neg_row[i];
  // device scratch: q rows, guesses, previous guesses, stable mask, found list + counter
  const int64_t cap = (int64_t)rounds * P;
  const size_t bytes = 8 * ((size_t)k + 1 + 2 * (size_t)P + (size_t)n_gwords + (size_t)cap + 1);
  if ((st = ensure(p, p->tune_in, bytes)) != LP_OK) return st;
  uint64_t* base = (uint64_t*)p->tune_in.p;
  int32_t* d_q = (int32_t*)base;
  uint64_t* d_guess = base + (k + 1) / 2 + 1;
  uint64_t* d_prev = d_guess + P;
  uint64_t* d_mask = d_prev + P;
  uint64_t* d_found = d_mask + n_gwords;
  unsigned long long* d_nfound = (unsigned long long*)(d_found + cap);
  LP_CUDA(cudaMemcpyAsync(d_q, qrow.data(), qrow.size() * 4, cudaMemcpyHostToDevice, s));
  LP_CUDA(cudaMemsetAsync(d_nfound, 0, 8, s));
  const int threads = 256, blocks = (P + threads - 1) / threads;
  search_init_kernel<<<blocks, threads, 0, s>>>(d_guess, d_prev, P, seed, kmask);
  if ((st = launch_count_and_check(cudaGetLastError(), "launch search init", p)) != LP_OK) return st;

  const lp_schedule saved = p->sched;
  p->sched.stable_tile_words = W;
  p->sched.stable_frontier = 0;  // the update reads the fixpoint from the full sweep's one tile
  for (int r = 0; r < rounds; r++) {
    st = lp_stable_models(p, d_guess, P, d_mask, nullptr, 0, nullptr, 1 << 30, cuda_stream);
    if (st != LP_OK) break;
    search_update_kernel<<<blocks, threads, 0, s>>>((const uint64_t*)p->tiles.p, __builtin_ctz((unsigned)W), d_q, k,
                                                    d_mask, d_guess, d_prev, P, seed, r, kmask, d_found, d_nfound,
                                                    cap);
    if ((st = launch_count_and_check(cudaGetLastError(), "launch search update", p)) != LP_OK) break;
  }
  p->sched = saved;
  if (st != LP_OK) return st;

  // distinct stable guesses, ascending
  unsigned long long total = 0;
  LP_CUDA(cudaMemcpyAsync(&total, d_nfound, 8, cudaMemcpyDeviceToHost, s));
  LP_CUDA(cudaStreamSynchronize(s));
  const int64_t got = std::min<int64_t>((int64_t)total, cap);
  std::vector<uint64_t> all((size_t)std::max<int64_t>(got, 1));
  if (got) LP_CUDA(cudaMemcpyAsync(all.data(), d_found, (size_t)got * 8, cudaMemcpyDeviceToHost, s));
  LP_CUDA(cudaStreamSynchronize(s));
  all.resize((size_t)got);
  std::sort(all.begin(), all.end());
  all.erase(std::unique(all.begin(), all.end()), all.end());
  *n_found = (int64_t)all.size();
  const int64_t out_n = std::min<int64_t>((int64_t)all.size(), max_found);
  if (out_n > 0) {
    LP_CUDA(cudaMemcpyAsync(found, all.data(), (size_t)out_n * 8, cudaMemcpyDefault, s));
    LP_CUDA(cudaStreamSynchronize(s));
  }
  return LP_OK;
}
