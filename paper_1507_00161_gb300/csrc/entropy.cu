// Two-orbital reduced density matrix of the dot orbitals p, p+1 of a two-site wave
// function: sums of products of wave-function elements over rectangular pieces of its
// blocks (occupation quadrants of the dots, and the pairs of pieces that a hop between
// two dots of equal quantum numbers connects).
//
// One warp per piece, lanes stride the piece's elements, fixed-order shuffle reduction;
// a single block then adds the pieces of each of the five sums in piece order.  FP64,
// deterministic for a fixed piece list.
#include <stdint.h>

#include "common.h"

namespace dmrg {

namespace {

constexpr int kRdmWarps = 8;
constexpr int kRdmSlots = 5;
constexpr int kRdmSumThreads = 256;

__global__ void __launch_bounds__(kRdmWarps * 32)
k_rdm_pieces(const RdmTask* __restrict__ tasks, int64_t n, const double* __restrict__ psi,
             double* __restrict__ part) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t w = int64_t(blockIdx.x) * kRdmWarps + warp; w < n;
       w += int64_t(gridDim.x) * kRdmWarps) {
    const RdmTask t = tasks[w];
    const int64_t cnt = int64_t(t.nr) * t.nc;
    double s = 0.0;
    for (int64_t e = lane; e < cnt; e += 32) {
      const int64_t i = e / t.nc, j = e - i * t.nc;
      s = fma(psi[t.a + i * t.lda + j], psi[t.b + i * t.ldb + j], s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) part[w] = s;
  }
}

__global__ void __launch_bounds__(kRdmSumThreads)
k_rdm_total(const RdmTask* __restrict__ tasks, int64_t n, const double* __restrict__ part,
            double* __restrict__ out) {
  __shared__ double sh[kRdmSlots][kRdmSumThreads];
  double acc[kRdmSlots] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int64_t i = threadIdx.x; i < n; i += kRdmSumThreads) {
    const int slot = tasks[i].slot;
#pragma unroll
    for (int k = 0; k < kRdmSlots; ++k)
      if (k == slot) acc[k] += part[i];
  }
#pragma unroll
  for (int k = 0; k < kRdmSlots; ++k) sh[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int h = kRdmSumThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h)
#pragma unroll
      for (int k = 0; k < kRdmSlots; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x < kRdmSlots) out[threadIdx.x] = sh[threadIdx.x][0];
}

}  // namespace

void rdm_sums(const RdmTask* d_tasks, int64_t n, const double* psi, double* d_part,
              double* d_out, cudaStream_t s) {
  if (n <= 0) {
    DMRG_CUDA(cudaMemsetAsync(d_out, 0, sizeof(double) * kRdmSlots, s));
    return;
  }
  const int64_t blocks = std::min<int64_t>((n + kRdmWarps - 1) / kRdmWarps, 152 * 16);
  k_rdm_pieces<<<int(blocks), kRdmWarps * 32, 0, s>>>(d_tasks, n, psi, d_part);
  DMRG_LAUNCHED();
  k_rdm_total<<<1, kRdmSumThreads, 0, s>>>(d_tasks, n, d_part, d_out);
  DMRG_LAUNCHED();
}

}  // namespace dmrg
