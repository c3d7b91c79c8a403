// relaxed.cu -- the relaxed (differentiable) fixpoint: forward, hand-written adjoint,
// checkpointing (lp_relaxed_* in include/lp.h).
//
// Each step replaces theta of Def. 5 by a sigmoid of temperature tau applied to the row sums
// x = M_P v of the program matrix (Def. 2/7), with a weight per rule row:
//   rule row of rule r, m body atoms:  u = sigmoid(w_r (x - 1 + 1/(2m)) / tau),  x = mean
//   OR-rule row:                       u = sigmoid((x - 1/2) / tau),             x = sum
//   self-loop (fact, barred atom):     u = v;      empty row: u = 0.
// With binary inputs and tau -> 0 this is theta exactly (|logit| >= w/(2 m tau)).
//
// Batches of b vectors are stored row-major, [row][b] floats, so a row's b values are
// contiguous: a warp handles one row and its lanes walk the batch, every gathered row is a
// coalesced read. The adjoint of one step, with g = dL/dv_{t+1} and e = g u (1 - u):
//   dL/dw_r += sum_batch e (x/m - 1 + 1/(2m)) / tau         (rule rows; float per 256 columns,
//                                                             double across passes and steps)
//   dL/dv_t  = M^T (c e) + g on self-loop rows,  c = w_r/(m tau) (rule), 1/tau (OR)
// where M^T is applied as a gather over a transposed copy (CSC) of the rule and OR rows. The
// column lengths of that copy follow the skew of the body atoms (a popular atom sits in 1e5
// rows), so every column's sum runs as a fixed reduction tree: chunks of up to 32 entries, then
// chunks of up to 32 partial sums, and so on. The tree depends only on the matrix, so results
// are the same bit for bit on every run, and no warp walks more than 32 rows.
// The forward keeps v every ckpt_every steps; the backward recomputes each segment from its
// checkpoint and runs the adjoint through it, last segment first.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "device.cuh"
#include "internal.h"
#include "kernels.h"
#include "program.h"

namespace lp {

enum RxKind : int { RX_RULE = 0, RX_OR = 1, RX_SELF = 2, RX_EMPTY = 3 };
constexpr int kRxBlock = 256;
constexpr int kRxPerLane = 8;  // batch values per lane per pass (256 columns per warp pass)

__device__ __forceinline__ float rx_sigmoid(float z) { return 1.0f / (1.0f + __expf(-z)); }

// A warp pass covers 256 batch columns, 8 per lane. Scalar layout (any b): slot k of a lane is
// column c0 + 32 k + lane. Vector layout (b a multiple of 4, 16-byte aligned rows): slots
// 4j..4j+3 are the float4 at column c0 + 128 j + 4 lane, so a warp moves 512 contiguous bytes
// per load instruction.
template <bool VEC>
__device__ __forceinline__ int rx_col(int c0, int lane, int k) {
  return VEC ? c0 + 128 * (k >> 2) + 4 * lane + (k & 3) : c0 + 32 * k + lane;
}

template <bool VEC>
__device__ __forceinline__ void rx_load(const float* row, int c0, int lane, int b, float (&v)[kRxPerLane]) {
  if (VEC) {
#pragma unroll
    for (int j = 0; j < kRxPerLane / 4; j++) {
      const int cb = c0 + 128 * j + 4 * lane;
      float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
      if (cb < b) q = *reinterpret_cast<const float4*>(row + cb);
      v[4 * j] = q.x;
      v[4 * j + 1] = q.y;
      v[4 * j + 2] = q.z;
      v[4 * j + 3] = q.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < kRxPerLane; k++) {
      const int c = c0 + 32 * k + lane;
      v[k] = c < b ? row[c] : 0.f;
    }
  }
}

template <bool VEC>
__device__ __forceinline__ void rx_store(float* row, int c0, int lane, int b, const float (&v)[kRxPerLane]) {
  if (VEC) {
#pragma unroll
    for (int j = 0; j < kRxPerLane / 4; j++) {
      const int cb = c0 + 128 * j + 4 * lane;
      if (cb < b) *reinterpret_cast<float4*>(row + cb) = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
    }
  } else {
#pragma unroll
    for (int k = 0; k < kRxPerLane; k++) {
      const int c = c0 + 32 * k + lane;
      if (c < b) row[c] = v[k];
    }
  }
}

template <bool VEC>
__global__ void __launch_bounds__(kRxBlock) rx_forward_kernel(const int32_t* __restrict__ row_ptr,
                                                              const int32_t* __restrict__ col,
                                                              const int32_t* __restrict__ info,
                                                              const int32_t* __restrict__ rule,
                                                              const float* __restrict__ w,
                                                              const float* __restrict__ vin,
                                                              float* __restrict__ vout, int n_rows, int b,
                                                              float inv_tau) {
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n_rows; i += nwarps) {
    const int inf = __ldg(info + i);
    const int kind = (int)((unsigned)inf >> 30);
    const int len = inf & 0x3fffffff;
    const int beg = __ldg(row_ptr + i);
    const size_t ro = (size_t)i * b;
    float wr = 0.f, inv_m = 0.f;
    if (kind == RX_RULE && len > 0) {
      wr = __ldg(w + __ldg(rule + i));
      inv_m = 1.0f / (float)len;
    }
    for (int c0 = 0; c0 < b; c0 += 32 * kRxPerLane) {
      float x[kRxPerLane], t[kRxPerLane];
#pragma unroll
      for (int k = 0; k < kRxPerLane; k++) x[k] = 0.f;
      if ((kind == RX_RULE || kind == RX_OR) && len > 0) {
        for (int e = 0; e < len; e++) {
          rx_load<VEC>(vin + (size_t)__ldg(col + beg + e) * b, c0, lane, b, t);
#pragma unroll
          for (int k = 0; k < kRxPerLane; k++) x[k] += t[k];
        }
      } else if (kind == RX_SELF) {
        rx_load<VEC>(vin + ro, c0, lane, b, x);
      }
#pragma unroll
      for (int k = 0; k < kRxPerLane; k++) {
        float u;
        if (kind == RX_SELF) u = x[k];
        else if (kind == RX_OR && len > 0) u = rx_sigmoid((x[k] - 0.5f) * inv_tau);
        else if (kind == RX_RULE && len > 0) u = rx_sigmoid(wr * (x[k] * inv_m - 1.0f + 0.5f * inv_m) * inv_tau);
        else u = 0.f;
        t[k] = u;
      }
      rx_store<VEC>(vout + ro, c0, lane, b, t);
    }
  }
}

// e_out = c * g * u (1 - u) for rule and OR rows; weight-gradient accumulation for rule rows.
template <bool VEC>
__global__ void __launch_bounds__(kRxBlock) rx_backward_rows_kernel(
    const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col, const int32_t* __restrict__ info,
    const int32_t* __restrict__ rule, const float* __restrict__ w, const float* __restrict__ vt,
    const float* __restrict__ u_t1, const float* __restrict__ g1, float* __restrict__ e_out, double* __restrict__ dw_row,
    int n_rows, int b, float inv_tau) {
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n_rows; i += nwarps) {
    const int inf = __ldg(info + i);
    const int kind = (int)((unsigned)inf >> 30);
    const int len = inf & 0x3fffffff;
    if (!((kind == RX_RULE || kind == RX_OR) && len > 0)) continue;  // no adjoint through these rows
    const int beg = __ldg(row_ptr + i);
    const size_t ro = (size_t)i * b;
    const bool is_rule = kind == RX_RULE;
    const float inv_m = is_rule ? 1.0f / (float)len : 1.0f;
    const float wr = is_rule ? __ldg(w + __ldg(rule + i)) : 1.0f;
    const float coef = is_rule ? wr * inv_m * inv_tau : inv_tau;
    // the row's weight gradient over the batch: float partial sums per 256-column pass (FP64
    // arithmetic is scarce on this part), accumulated in double across passes and steps
    double dsum = 0.0;
    for (int c0 = 0; c0 < b; c0 += 32 * kRxPerLane) {
      float x[kRxPerLane], t[kRxPerLane], u[kRxPerLane], g[kRxPerLane];
      float fsum = 0.0f;
#pragma unroll
      for (int k = 0; k < kRxPerLane; k++) x[k] = 0.f;
      if (is_rule) {  // the row sum again (for the weight gradient)
        for (int e = 0; e < len; e++) {
          rx_load<VEC>(vt + (size_t)__ldg(col + beg + e) * b, c0, lane, b, t);
#pragma unroll
          for (int k = 0; k < kRxPerLane; k++) x[k] += t[k];
        }
      }
      rx_load<VEC>(u_t1 + ro, c0, lane, b, u);
      rx_load<VEC>(g1 + ro, c0, lane, b, g);
#pragma unroll
      for (int k = 0; k < kRxPerLane; k++) {
        const float e = g[k] * u[k] * (1.0f - u[k]);
        t[k] = coef * e;
        if (is_rule && rx_col<VEC>(c0, lane, k) < b) fsum += e * (x[k] * inv_m - 1.0f + 0.5f * inv_m);
      }
      rx_store<VEC>(e_out + ro, c0, lane, b, t);
      if (is_rule) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) fsum += __shfl_xor_sync(FULL, fsum, o);
        dsum += (double)fsum;
      }
    }
    if (is_rule && lane == 0) dw_row[i] += dsum * (double)inv_tau;
  }
}

// One node of the reduction tree of g0 = M^T e: the sum of `count` source rows of b floats,
// from e rows listed in the transpose (level 0: rowidx[src ..]) or from consecutive partial rows
// of the previous level (partial rows src ..). dst >= 0: a partial row of this level's output;
// dst < 0: the final value of column j, plus g1[j] on a self-loop row.
struct RxUnit {
  int64_t src;
  int64_t dst;
  int32_t j;
  int32_t count;
};
constexpr int kRxFan = 32;  // children per tree node

template <bool VEC>
__global__ void __launch_bounds__(kRxBlock) rx_reduce_kernel(const RxUnit* __restrict__ units, int64_t n_units,
                                                             const int32_t* __restrict__ rowidx,
                                                             const float* __restrict__ src,
                                                             float* __restrict__ part_out,
                                                             const int32_t* __restrict__ info,
                                                             const float* __restrict__ g1,
                                                             float* __restrict__ g0, int b) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n_units; u += nwarps) {
    const RxUnit un = units[u];
    const bool fin = un.dst < 0;
    const bool self = fin && (int)((unsigned)__ldg(info + un.j) >> 30) == RX_SELF;
    float* out = fin ? g0 + (size_t)un.j * b : part_out + (size_t)un.dst * b;
    for (int c0 = 0; c0 < b; c0 += 32 * kRxPerLane) {
      float acc[kRxPerLane], t[kRxPerLane];
      if (self) {
        rx_load<VEC>(g1 + (size_t)un.j * b, c0, lane, b, acc);
      } else {
#pragma unroll
        for (int k = 0; k < kRxPerLane; k++) acc[k] = 0.f;
      }
      for (int q = 0; q < un.count; q++) {
        const size_t r = rowidx ? (size_t)__ldg(rowidx + un.src + q) : (size_t)(un.src + q);
        rx_load<VEC>(src + r * b, c0, lane, b, t);
#pragma unroll
        for (int k = 0; k < kRxPerLane; k++) acc[k] += t[k];
      }
      rx_store<VEC>(out, c0, lane, b, acc);
    }
  }
}

// Canonical <-> internal row order of [row][b] arrays, one warp per destination row: row r of
// dst is row map[r] of src (to internal: map = internal -> canonical, rows past n_src are zero;
// to canonical: map = canonical -> internal).
template <bool VEC>
__global__ void __launch_bounds__(kRxBlock) rx_permute_rows_kernel(const float* __restrict__ src,
                                                                   float* __restrict__ dst,
                                                                   const int32_t* __restrict__ map, int n_src,
                                                                   int n_dst, int b) {
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n_dst; r += nwarps) {
    const bool live = r < n_src;
    const float* from = live ? src + (size_t)__ldg(map + r) * b : nullptr;
    float* to = dst + (size_t)r * b;
    for (int c0 = 0; c0 < b; c0 += 32 * kRxPerLane) {
      float v[kRxPerLane];
      if (live) {
        rx_load<VEC>(from, c0, lane, b, v);
      } else {
#pragma unroll
        for (int k = 0; k < kRxPerLane; k++) v[k] = 0.f;
      }
      rx_store<VEC>(to, c0, lane, b, v);
    }
  }
}

__global__ void rx_dw_out_kernel(const double* __restrict__ dw_row, const int32_t* __restrict__ rule,
                                 float* __restrict__ dw, int n_rows) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_rows; i += gridDim.x * blockDim.x) {
    const int r = __ldg(rule + i);
    if (r >= 0) dw[r] = (float)dw_row[i];
  }
}

namespace {

int rx_grid(lp_program* p, int64_t warps_needed) {
  const int64_t blocks = (warps_needed * 32 + kRxBlock - 1) / kRxBlock;
  return (int)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)p->sm_count * 16));
}

// Builds the per-row kinds, rule ids and the transposed copy on first use.
lp_status ensure_relaxed(lp_program* p, cudaStream_t s) {
  if (p->rx_ready) return LP_OK;
  const lp_status ht = ensure_host_tables(p, s);
  if (ht != LP_OK) return ht;
  const HostMatrix& hm = p->hm;
  std::vector<int32_t> rp((size_t)hm.n_pad + 1), cl(std::max<int64_t>(hm.nnz, 1));
  LP_CUDA(cudaMemcpyAsync(rp.data(), p->row_ptr, rp.size() * 4, cudaMemcpyDeviceToHost, s));
  if (hm.nnz) LP_CUDA(cudaMemcpyAsync(cl.data(), p->col, (size_t)hm.nnz * 4, cudaMemcpyDeviceToHost, s));
  LP_CUDA(cudaStreamSynchronize(s));
  std::vector<int32_t> info(hm.n_pad, (int32_t)((unsigned)RX_EMPTY << 30)), rule(hm.n_pad, -1);
  for (int32_t c = 0; c < hm.n_prime; c++) {
    const int32_t r = hm.perm[c];
    const int32_t len = rp[r + 1] - rp[r];
    int kind;
    switch (hm.canon_kind[c]) {
      case K_RULE: kind = RX_RULE; break;
      case K_OR: kind = RX_OR; break;
      case K_FACT:
      case K_BARRED: kind = RX_SELF; break;
      default: kind = RX_EMPTY; break;
    }
    info[r] = (int32_t)(((unsigned)kind << 30) | (unsigned)len);
    rule[r] = hm.canon_rule[c];
  }
  // transpose of the rule and OR rows (self-loops pass their gradient through directly)
  std::vector<int32_t> cp((size_t)hm.n_pad + 1, 0);
  for (int32_t r = 0; r < hm.n_pad; r++) {
    const int kind = (int)((unsigned)info[r] >> 30);
    if (kind == RX_RULE || kind == RX_OR)
      for (int32_t e = rp[r]; e < rp[r + 1]; e++) cp[cl[e] + 1]++;
  }
  for (int32_t j = 0; j < hm.n_pad; j++) cp[j + 1] += cp[j];
  std::vector<int32_t> ri(std::max<int32_t>(cp[hm.n_pad], 1));
  {
    std::vector<int32_t> cur(cp.begin(), cp.end() - 1);
    for (int32_t r = 0; r < hm.n_pad; r++) {
      const int kind = (int)((unsigned)info[r] >> 30);
      if (kind == RX_RULE || kind == RX_OR)
        for (int32_t e = rp[r]; e < rp[r + 1]; e++) ri[cur[cl[e]]++] = r;
    }
  }
  // reduction tree of every column: level 0 sums chunks of <= kRxFan transpose entries; a
  // column with more than one chunk continues at the next level over its chunks' partial rows
  std::vector<RxUnit> units;
  p->rx_level_off.assign(1, 0);
  p->rx_part_off.assign(1, 0);
  struct Pending {
    int32_t j;
    int64_t first, n;  // partial rows [first, first + n) of the previous level
  };
  std::vector<Pending> pend, next_pend;
  int64_t part = 0;
  for (int32_t j = 0; j < hm.n_pad; j++) {
    const int64_t deg = cp[j + 1] - cp[j];
    if (deg <= kRxFan) {
      units.push_back({cp[j], -1, j, (int32_t)deg});
      continue;
    }
    const int64_t first = part;
    for (int64_t c = 0; c < deg; c += kRxFan)
      units.push_back({cp[j] + c, part++, j, (int32_t)std::min<int64_t>(kRxFan, deg - c)});
    pend.push_back({j, first, part - first});
  }
  p->rx_level_off.push_back((int64_t)units.size());
  p->rx_part_off.push_back(part);
  while (!pend.empty()) {
    next_pend.clear();
    for (const Pending& q : pend) {
      if (q.n <= kRxFan) {
        units.push_back({q.first, -1, q.j, (int32_t)q.n});
        continue;
      }
      const int64_t first = part;
      for (int64_t c = 0; c < q.n; c += kRxFan)
        units.push_back({q.first + c, part++, q.j, (int32_t)std::min<int64_t>(kRxFan, q.n - c)});
      next_pend.push_back({q.j, first, part - first});
    }
    p->rx_level_off.push_back((int64_t)units.size());
    p->rx_part_off.push_back(part);
    pend.swap(next_pend);
  }
  lp_status st;
  if ((st = upload(p, reinterpret_cast<RxUnit**>(&p->rx_units), units, s)) != LP_OK) return st;
  if ((st = upload(p, &p->rx_info, info, s)) != LP_OK) return st;
  if ((st = upload(p, &p->rx_rule, rule, s)) != LP_OK) return st;
  if ((st = upload(p, &p->rx_rowidx, ri, s)) != LP_OK) return st;
  if ((st = ensure(p, p->rx_dw, (size_t)hm.n_pad * sizeof(double))) != LP_OK) return st;
  LP_CUDA(cudaStreamSynchronize(s));
  p->rx_ready = true;
  return LP_OK;
}

lp_status rx_check(lp_program* p, int32_t b, int32_t steps, float tau, int32_t ckpt_every) {
  if (!p) return fail(LP_ERR_INVALID, "program must not be NULL");
  if (p->host_only) return fail(LP_ERR_INVALID, "program was compiled with LP_COMPILE_HOST_ONLY");
  if (b < 1 || steps < 1 || ckpt_every < 1) return fail(LP_ERR_INVALID, "batch, steps and ckpt_every must be >= 1");
  if (!(tau > 0.0f)) return fail(LP_ERR_INVALID, "tau must be > 0");
  return LP_OK;
}

lp_status rx_launched(cudaError_t e, lp_program* p) { return launch_count_and_check(e, "launch relaxed kernel", p); }

// float4 row access: every [row][b] buffer the kernels touch starts at base + a multiple of
// n_pad * b floats, so b % 4 == 0 and a 16-byte aligned base keep every row 16-byte aligned
bool vec_rows(int32_t b, const void* base) { return b % 4 == 0 && ((uintptr_t)base & 15u) == 0; }

}  // namespace
}  // namespace lp

using namespace lp;

extern "C" {

lp_status lp_relaxed_workspace(lp_program* p, int32_t batch, int32_t steps, int32_t ckpt_every, int64_t* ckpt_floats,
                               int64_t* scratch_floats) {
  lp_status st = rx_check(p, batch, steps, 1.0f, ckpt_every);
  if (st != LP_OK) return st;
  const int64_t nb = (int64_t)p->hm.n_pad * batch;
  const int64_t n_ckpt = (steps + ckpt_every - 1) / ckpt_every;
  if (ckpt_floats) *ckpt_floats = (n_ckpt + 2) * nb;
  if (scratch_floats) *scratch_floats = ((int64_t)ckpt_every + 3) * nb;
  return LP_OK;
}

lp_status lp_relaxed_forward(lp_program* p, const float* weights, const float* v0, int32_t batch, int32_t steps,
                             float tau, int32_t ckpt_every, float* ckpt, float* vT, void* cuda_stream) {
  NvtxRange nvtx("lp_relaxed_forward");
  lp_status st = rx_check(p, batch, steps, tau, ckpt_every);
  if (st != LP_OK) return st;
  if (!weights || !v0 || !ckpt || !vT) return fail(LP_ERR_INVALID, "NULL buffer");
  if (!is_device_ptr(weights) || !is_device_ptr(v0) || !is_device_ptr(ckpt) || !is_device_ptr(vT))
    return fail(LP_ERR_INVALID, "relaxed buffers must be device memory");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if ((st = ensure_relaxed(p, s)) != LP_OK) return st;
  p->last_launches = 0;
  const HostMatrix& hm = p->hm;
  if (!p->inv) {
    std::vector<int32_t> inv(std::max(hm.n_pad, 1), 0);
    for (int32_t c = 0; c < hm.n_prime; c++) inv[hm.perm[c]] = c;
    if ((st = upload(p, &p->inv, inv, s)) != LP_OK) return st;
    LP_CUDA(cudaStreamSynchronize(s));
  }
  const size_t nb = (size_t)hm.n_pad * batch;
  const int n_ckpt = (steps + ckpt_every - 1) / ckpt_every;
  float* tmp0 = ckpt + (size_t)n_ckpt * nb;
  float* tmp1 = tmp0 + nb;
  const float inv_tau = 1.0f / tau;
  const int rg = rx_grid(p, hm.n_pad);
  const bool vec = vec_rows(batch, ckpt);
  const bool vec_io = vec && vec_rows(batch, v0) && vec_rows(batch, vT);
  if (vec_io) rx_permute_rows_kernel<true><<<rg, kRxBlock, 0, s>>>(v0, ckpt, p->inv, hm.n_prime, hm.n_pad, batch);
  else rx_permute_rows_kernel<false><<<rg, kRxBlock, 0, s>>>(v0, ckpt, p->inv, hm.n_prime, hm.n_pad, batch);
  if ((st = rx_launched(cudaGetLastError(), p)) != LP_OK) return st;
  float* cur = ckpt;
  for (int t = 0; t < steps; t++) {
    float* next = ((t + 1) % ckpt_every == 0 && t + 1 < steps) ? ckpt + (size_t)((t + 1) / ckpt_every) * nb
                                                                : (cur == tmp0 ? tmp1 : tmp0);
    if (vec)
      rx_forward_kernel<true><<<rg, kRxBlock, 0, s>>>(p->row_ptr, p->col, p->rx_info, p->rx_rule, weights, cur, next,
                                                      hm.n_pad, batch, inv_tau);
    else
      rx_forward_kernel<false><<<rg, kRxBlock, 0, s>>>(p->row_ptr, p->col, p->rx_info, p->rx_rule, weights, cur,
                                                       next, hm.n_pad, batch, inv_tau);
    if ((st = rx_launched(cudaGetLastError(), p)) != LP_OK) return st;
    cur = next;
  }
  if (vec_io) rx_permute_rows_kernel<true><<<rg, kRxBlock, 0, s>>>(cur, vT, p->perm, hm.n_prime, hm.n_prime, batch);
  else rx_permute_rows_kernel<false><<<rg, kRxBlock, 0, s>>>(cur, vT, p->perm, hm.n_prime, hm.n_prime, batch);
  return rx_launched(cudaGetLastError(), p);
}

lp_status lp_relaxed_backward(lp_program* p, const float* weights, const float* gT, int32_t batch, int32_t steps,
                              float tau, int32_t ckpt_every, const float* ckpt, float* scratch, float* dweights,
                              float* dv0, void* cuda_stream) {
  NvtxRange nvtx("lp_relaxed_backward");
  lp_status st = rx_check(p, batch, steps, tau, ckpt_every);
  if (st != LP_OK) return st;
  if (!weights || !gT || !ckpt || !scratch || !dweights || !dv0) return fail(LP_ERR_INVALID, "NULL buffer");
  if (!is_device_ptr(weights) || !is_device_ptr(gT) || !is_device_ptr(ckpt) || !is_device_ptr(scratch) ||
      !is_device_ptr(dweights) || !is_device_ptr(dv0))
    return fail(LP_ERR_INVALID, "relaxed buffers must be device memory");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if ((st = ensure_relaxed(p, s)) != LP_OK) return st;
  if (!p->inv) return fail(LP_ERR_INVALID, "lp_relaxed_backward needs a preceding lp_relaxed_forward");
  p->last_launches = 0;
  const HostMatrix& hm = p->hm;
  const size_t nb = (size_t)hm.n_pad * batch;
  const int n_ckpt = (steps + ckpt_every - 1) / ckpt_every;
  float* seg = scratch;  // ckpt_every states of the current segment
  float* E = scratch + (size_t)ckpt_every * nb;
  float* G0 = E + nb;
  float* G1 = G0 + nb;
  const float inv_tau = 1.0f / tau;
  const int rg = rx_grid(p, hm.n_pad);
  const bool vec = vec_rows(batch, ckpt) && vec_rows(batch, scratch);
  if ((st = ensure(p, p->rx_part, std::max<size_t>((size_t)p->rx_part_off.back() * batch * sizeof(float), 4))) !=
      LP_OK)
    return st;
  LP_CUDA(cudaMemsetAsync(p->rx_dw.p, 0, (size_t)hm.n_pad * sizeof(double), s));
  const bool vec_io = vec && vec_rows(batch, gT) && vec_rows(batch, dv0);
  if (vec_io) rx_permute_rows_kernel<true><<<rg, kRxBlock, 0, s>>>(gT, G0, p->inv, hm.n_prime, hm.n_pad, batch);
  else rx_permute_rows_kernel<false><<<rg, kRxBlock, 0, s>>>(gT, G0, p->inv, hm.n_prime, hm.n_pad, batch);
  if ((st = rx_launched(cudaGetLastError(), p)) != LP_OK) return st;
  float* g = G0;
  for (int c = n_ckpt - 1; c >= 0; c--) {
    const int t0 = c * ckpt_every, t1 = std::min(t0 + ckpt_every, (int)steps);
    const float* prev = ckpt + (size_t)c * nb;
    for (int t = t0; t < t1; t++) {  // recompute v_{t0+1} .. v_{t1}
      float* next = seg + (size_t)(t - t0) * nb;
      if (vec)
        rx_forward_kernel<true><<<rg, kRxBlock, 0, s>>>(p->row_ptr, p->col, p->rx_info, p->rx_rule, weights, prev,
                                                        next, hm.n_pad, batch, inv_tau);
      else
        rx_forward_kernel<false><<<rg, kRxBlock, 0, s>>>(p->row_ptr, p->col, p->rx_info, p->rx_rule, weights, prev,
                                                         next, hm.n_pad, batch, inv_tau);
      if ((st = rx_launched(cudaGetLastError(), p)) != LP_OK) return st;
      prev = next;
    }
    for (int t = t1 - 1; t >= t0; t--) {
      const float* vt = (t == t0) ? ckpt + (size_t)c * nb : seg + (size_t)(t - t0 - 1) * nb;
      const float* vt1 = seg + (size_t)(t - t0) * nb;
      if (vec)
        rx_backward_rows_kernel<true><<<rg, kRxBlock, 0, s>>>(p->row_ptr, p->col, p->rx_info, p->rx_rule, weights, vt,
                                                              vt1, g, E, (double*)p->rx_dw.p, hm.n_pad, batch,
                                                              inv_tau);
      else
        rx_backward_rows_kernel<false><<<rg, kRxBlock, 0, s>>>(p->row_ptr, p->col, p->rx_info, p->rx_rule, weights,
                                                               vt, vt1, g, E, (double*)p->rx_dw.p, hm.n_pad, batch,
                                                               inv_tau);
      if ((st = rx_launched(cudaGetLastError(), p)) != LP_OK) return st;
      float* gn = (g == G0) ? G1 : G0;
      // g_t = M^T E (+ g on self-loops), level by level; partial rows are numbered across all
      // levels (level L writes rows [rx_part_off[L], rx_part_off[L + 1]), level L + 1 reads them)
      const RxUnit* units = reinterpret_cast<const RxUnit*>(p->rx_units);
      float* part = (float*)p->rx_part.p;
      const int n_levels = (int)p->rx_level_off.size() - 1;
      for (int L = 0; L < n_levels; L++) {
        const int64_t u0 = p->rx_level_off[L], nu = p->rx_level_off[L + 1] - u0;
        if (nu == 0) continue;
        if (vec)
          rx_reduce_kernel<true><<<rx_grid(p, nu), kRxBlock, 0, s>>>(units + u0, nu, L == 0 ? p->rx_rowidx : nullptr,
                                                                     L == 0 ? E : part, part, p->rx_info, g, gn, batch);
        else
          rx_reduce_kernel<false><<<rx_grid(p, nu), kRxBlock, 0, s>>>(units + u0, nu, L == 0 ? p->rx_rowidx : nullptr,
                                                                      L == 0 ? E : part, part, p->rx_info, g, gn,
                                                                      batch);
        if ((st = rx_launched(cudaGetLastError(), p)) != LP_OK) return st;
      }
      g = gn;
    }
  }
  if (vec_io) rx_permute_rows_kernel<true><<<rg, kRxBlock, 0, s>>>(g, dv0, p->perm, hm.n_prime, hm.n_prime, batch);
  else rx_permute_rows_kernel<false><<<rg, kRxBlock, 0, s>>>(g, dv0, p->perm, hm.n_prime, hm.n_prime, batch);
  if ((st = rx_launched(cudaGetLastError(), p)) != LP_OK) return st;
  LP_CUDA(cudaMemsetAsync(dweights, 0, (size_t)std::max<int64_t>(hm.n_rules, 0) * sizeof(float), s));
  rx_dw_out_kernel<<<rg, kRxBlock, 0, s>>>((const double*)p->rx_dw.p, p->rx_rule, dweights, hm.n_pad);
  return rx_launched(cudaGetLastError(), p);
}

}  // extern "C"
