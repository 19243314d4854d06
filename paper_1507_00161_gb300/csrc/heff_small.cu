// Superblock product for small blocks:  psi'(b') += s_k L_k psi(b) R_k^T  (the two-site
// H_eff of the superblock "Xi_l (x) Lambda (x) Lambda (x) Xi_r") for output blocks whose
// dimensions and whose terms' inner dimensions are all at most 16.
//
// At large M the sector count grows with M, so most wave-function blocks are a few states
// on a side: a term is a handful of multiply-adds and the work is streaming the operator
// blocks.  One warp per (output block, group of at most 16 terms), plain FMAs on the CUDA
// cores, operands read through the L1 (no staging, no padding to matrix-instruction shapes).
// Lane map for an m x n output block: column c = lane mod n, row group g = lane / n,
// G = floor(32 / n) groups; per term
//     X[a][c] = sum_b psi[a][b] R[c][b]   (rows a = g, g + G, ...; X in shared memory)
//     acc[i][c] += s sum_a L[i][a] X[a][c] (rows i = g, g + G, ...; acc in registers)
// Terms are added in list order; groups of one block are added in group order by
// k_heff_reduce: the result is deterministic.
#include <stdint.h>

#include "common.h"

namespace dmrg {

namespace {

constexpr int kSmWarps = 8;

template <class T>
__global__ void __launch_bounds__(kSmWarps * 32, 3)
k_heff_small(const HeffTile* __restrict__ tiles, int64_t n_tiles,
             const HeffItem* __restrict__ items, const HeffPtrs<T> ptrs) {
  __shared__ T Xs[kSmWarps][kSmallEdge * kSmallEdge];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* Xw = Xs[warp];
  for (int64_t w = int64_t(blockIdx.x) * kSmWarps + warp; w < n_tiles;
       w += int64_t(gridDim.x) * kSmWarps) {
    const HeffTile t = tiles[w];
    if (ptrs.active && !ptrs.active[t.inst]) continue;
    const T* __restrict__ L = ptrs.L[t.inst];
    const T* __restrict__ R = ptrs.R[t.inst];
    const T* __restrict__ X = ptrs.X[t.inst];
    const int m = t.m, n = t.n;
    const int G = 32 / n;
    const int c = lane % n, g = lane / n;
    const bool on = g < G;
    T acc[kSmallEdge / 2];
#pragma unroll
    for (int q = 0; q < kSmallEdge / 2; ++q) acc[q] = T(0);
    for (int base = t.i0; base < t.i1; base += 32) {
      // the lanes load the next 32 term descriptors at once; each term broadcasts its own
      HeffItem mine{};
      if (base + lane < t.i1) mine = items[base + lane];
      const int cnt = min(32, t.i1 - base);
      for (int j = 0; j < cnt; ++j) {
        const int64_t loff = __shfl_sync(0xffffffffu, (long long)mine.loff, j);
        const int64_t roff = __shfl_sync(0xffffffffu, (long long)mine.roff, j);
        const int64_t xoff = __shfl_sync(0xffffffffu, (long long)mine.xoff, j);
        const int dLi = __shfl_sync(0xffffffffu, mine.dLi, j);
        const int dRi = __shfl_sync(0xffffffffu, mine.dRi, j);
        const float sign = __shfl_sync(0xffffffffu, mine.sign, j);
        const T* __restrict__ Lb = L + loff + int64_t(t.r0) * dLi;
        const T* __restrict__ Rb = R + roff + int64_t(t.c0 + c) * dRi;
        const T* __restrict__ Xb = X + xoff;
        if (on) {
          for (int a = g; a < dLi; a += G) {
            T s = T(0);
            for (int b = 0; b < dRi; ++b) s = fma(Xb[a * dRi + b], Rb[b], s);
            Xw[a * n + c] = s;
          }
        }
        __syncwarp();
        if (on) {
          const T sg = T(sign);
#pragma unroll
          for (int q = 0; q < kSmallEdge / 2; ++q) {
            const int i = g + q * G;
            if (i < m) {
              T s = T(0);
              for (int a = 0; a < dLi; ++a) s = fma(Lb[i * dLi + a], Xw[a * n + c], s);
              acc[q] = fma(sg, s, acc[q]);
            }
          }
        }
        __syncwarp();
      }
    }
    if (on) {
      if (t.poff < 0) {
        T* __restrict__ Y = ptrs.Y[t.inst] + t.yoff;
#pragma unroll
        for (int q = 0; q < kSmallEdge / 2; ++q) {
          const int i = g + q * G;
          if (i < m) Y[int64_t(t.r0 + i) * t.ld + t.c0 + c] = acc[q];
        }
      } else {
        T* __restrict__ P = ptrs.P[t.inst] + t.poff;
#pragma unroll
        for (int q = 0; q < kSmallEdge / 2; ++q) {
          const int i = g + q * G;
          if (i < m) P[i * n + c] = acc[q];
        }
      }
    }
  }
}

}  // namespace

template <class T>
void heff_small(const HeffTile* d_tiles, int64_t n_tiles, const HeffItem* d_items,
                const HeffPtrs<T>& ptrs, cudaStream_t s) {
  if (n_tiles <= 0) return;
  const int64_t blocks = std::min<int64_t>((n_tiles + kSmWarps - 1) / kSmWarps, 152 * 8 * 16);
  k_heff_small<T><<<int(blocks), kSmWarps * 32, 0, s>>>(d_tiles, n_tiles, d_items, ptrs);
  DMRG_LAUNCHED();
}
template void heff_small<float>(const HeffTile*, int64_t, const HeffItem*, const HeffPtrs<float>&,
                                cudaStream_t);
template void heff_small<double>(const HeffTile*, int64_t, const HeffItem*,
                                 const HeffPtrs<double>&, cudaStream_t);

}  // namespace dmrg
