// Kernels of the all-pairs orbital mutual information (the entropy and mutual-information
// analysis that the ordering of the orbitals is chosen from):
//   * rect_dots: sign * sum_ij A[a + i lda + j] B[b + i ldb + j] over rectangles (an
//     operator block of the left block against a piece of a density or transition matrix
//     of the wave function), or the trace of the B rectangle (lda < 0: identity operator);
//     one warp per rectangle, fixed-order shuffle reduction;
//   * slot_sums: the rectangles of each slot added in list order (one thread per slot);
//   * embed_blocks: copy of a sub-block (or an identity) with a sign into an operator
//     block of the enlarged space (the carried operators before their renormalization).
// FP64 and deterministic for a fixed task list.
#include <stdint.h>

#include "common.h"

namespace dmrg {

namespace {

constexpr int kDotWarps = 8;

__global__ void __launch_bounds__(kDotWarps * 32)
k_rect_dots(const RectDot* __restrict__ tasks, int64_t n, const double* __restrict__ A,
            const double* __restrict__ B, double* __restrict__ part) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t w = int64_t(blockIdx.x) * kDotWarps + warp; w < n;
       w += int64_t(gridDim.x) * kDotWarps) {
    const RectDot t = tasks[w];
    double s = 0.0;
    if (t.lda < 0) {   // trace of the B rectangle (square)
      for (int i = lane; i < t.nr; i += 32) s += B[t.b + int64_t(i) * t.ldb + i];
    } else {
      const int64_t cnt = int64_t(t.nr) * t.nc;
      for (int64_t e = lane; e < cnt; e += 32) {
        const int64_t i = e / t.nc, j = e - i * t.nc;
        s = fma(A[t.a + i * t.lda + j], B[t.b + i * t.ldb + j], s);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) part[w] = t.sign * s;
  }
}

__global__ void k_slot_sums(const int64_t* __restrict__ ptr, int64_t n_slots,
                            const double* __restrict__ part, double* __restrict__ out) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= n_slots) return;
  double s = 0.0;
  for (int64_t t = ptr[k]; t < ptr[k + 1]; ++t) s += part[t];
  out[k] = s;
}

__global__ void k_embed(const EmbedTask* __restrict__ tasks, int64_t n,
                        const double* __restrict__ S, double* __restrict__ D) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t w = int64_t(blockIdx.x) * kDotWarps + warp; w < n;
       w += int64_t(gridDim.x) * kDotWarps) {
    const EmbedTask t = tasks[w];
    const int64_t cnt = int64_t(t.nr) * t.nc;
    for (int64_t e = lane; e < cnt; e += 32) {
      const int64_t i = e / t.nc, j = e - i * t.nc;
      const double v = t.src >= 0 ? S[t.src + i * t.lds + j] : (i == j ? 1.0 : 0.0);
      D[t.dst + i * t.ldd + j] = t.sign * v;
    }
  }
}

int grid_warps(int64_t n) {
  return int(std::max<int64_t>(1, std::min<int64_t>((n + kDotWarps - 1) / kDotWarps, 152 * 16)));
}

}  // namespace

void rect_dots(const RectDot* d_tasks, int64_t n, const double* A, const double* B,
               double* d_part, cudaStream_t s) {
  if (n <= 0) return;
  k_rect_dots<<<grid_warps(n), kDotWarps * 32, 0, s>>>(d_tasks, n, A, B, d_part);
  DMRG_LAUNCHED();
}

void slot_sums(const int64_t* d_ptr, int64_t n_slots, const double* d_part, double* d_out,
               cudaStream_t s) {
  if (n_slots <= 0) return;
  k_slot_sums<<<int((n_slots + 127) / 128), 128, 0, s>>>(d_ptr, n_slots, d_part, d_out);
  DMRG_LAUNCHED();
}

void embed_blocks(const EmbedTask* d_tasks, int64_t n, const double* S, double* D,
                  cudaStream_t s) {
  if (n <= 0) return;
  k_embed<<<grid_warps(n), kDotWarps * 32, 0, s>>>(d_tasks, n, S, D);
  DMRG_LAUNCHED();
}

}  // namespace dmrg
