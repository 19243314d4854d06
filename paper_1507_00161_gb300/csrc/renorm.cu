// Renormalization of block operators onto the kept states (the block basis update after
// the density-matrix truncation):  O'[n_o, n_i] = U_o^T  O[Q_o, Q_i]  U_i  for every block
// of every normal and complementary operator, U_Q = kept eigenvectors of the reduced
// density matrix in enlarged sector Q (D_Q x m_Q, row-major).
//
// Driven by the block table itself (no per-GEMM task lists):
//  - blocks with D_o, D_i <= 32: one warp each, both products fused, T = O U_i held in
//    shared memory; lane = (column c, row group g) so that narrow blocks keep all lanes busy;
//  - larger blocks: two batched GEMM passes, T_b = O_b U_i to a scratch, then
//    O'_b = U_o^T T_b, each cut into 32 x 32 output tiles; thread block t finds its block by
//    binary search in the prefix sums of tiles per block; K in chunks of 32 through shared
//    memory.
// FP64 throughout, fixed summation order (deterministic).
#include <stdint.h>

#include "common.h"

namespace dmrg {

namespace {

constexpr int kPT = 32;              // tile edge
constexpr int kPS = kPT + 1;         // padded shared row
constexpr int kPThreads = 128;

// C (M x N, ldc) = op(A) (M x K) B (K x N, ldb); A stored M x K (lda) or, transposed, K x M
// (lda).  Thread (ty, tx) owns rows ty, ty + 16 and columns tx, tx + 8, tx + 16, tx + 24.
template <bool TA>
__device__ __forceinline__ void tile_gemm(const double* __restrict__ A, int lda,
                                          const double* __restrict__ B, int ldb,
                                          double* __restrict__ C, int ldc, int M, int N, int K,
                                          int r0, int c0, double (*As)[kPS], double (*Bs)[kPS]) {
  const int tid = threadIdx.x;
  const int ty = tid >> 3, tx = tid & 7;
  double acc[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
  for (int k0 = 0; k0 < K; k0 += kPT) {
    for (int e = tid; e < kPT * kPT; e += kPThreads) {
      const int i = e >> 5, j = e & 31;
      if (TA)   // As[k][row] = A^T: A stored K x M
        As[i][j] = (k0 + i < K && r0 + j < M) ? A[int64_t(k0 + i) * lda + r0 + j] : 0.0;
      else      // As[row][k]
        As[i][j] = (r0 + i < M && k0 + j < K) ? A[int64_t(r0 + i) * lda + k0 + j] : 0.0;
      Bs[i][j] = (k0 + i < K && c0 + j < N) ? B[int64_t(k0 + i) * ldb + c0 + j] : 0.0;
    }
    __syncthreads();
    const int kn = min(kPT, K - k0);
#pragma unroll 4
    for (int k = 0; k < kn; ++k) {
      const double a0 = TA ? As[k][ty] : As[ty][k];
      const double a1 = TA ? As[k][ty + 16] : As[ty + 16][k];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const double b = Bs[k][tx + 8 * q];
        acc[0][q] = fma(a0, b, acc[0][q]);
        acc[1][q] = fma(a1, b, acc[1][q]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = r0 + ty + 16 * h, cc = c0 + tx + 8 * q;
      if (r < M && cc < N) C[int64_t(r) * ldc + cc] = acc[h][q];
    }
}

template <int STAGE>
__global__ void __launch_bounds__(kPThreads)
k_project(const ProjTask* __restrict__ tasks, const int64_t* __restrict__ tile_beg, int64_t n,
          const int32_t* __restrict__ D, const int32_t* __restrict__ m,
          const int64_t* __restrict__ uoff, const double* __restrict__ X,
          const double* __restrict__ U, double* __restrict__ T, double* __restrict__ Y) {
  __shared__ double As[kPT][kPS];
  __shared__ double Bs[kPT][kPS];
  const int64_t n_tiles = tile_beg[n];
  for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    // block b: tile_beg[b] <= t < tile_beg[b + 1]
    int64_t lo = 0, hi = n;
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) >> 1;
      if (tile_beg[mid] <= t) lo = mid;
      else hi = mid;
    }
    const ProjTask pt = tasks[lo];
    const int l = int(t - tile_beg[lo]);
    const int Do = D[pt.so], Di = D[pt.si], mo = m[pt.so], mi = m[pt.si];
    const int nct = (mi + kPT - 1) / kPT;
    const int r0 = (l / nct) * kPT, c0 = (l % nct) * kPT;
    if (STAGE == 1)
      tile_gemm<false>(X + pt.xoff, Di, U + uoff[pt.si], mi, T + pt.toff, mi, Do, mi, Di, r0, c0,
                       As, Bs);
    else
      tile_gemm<true>(U + uoff[pt.so], mo, T + pt.toff, mi, Y + pt.yoff, mi, mo, mi, Do, r0, c0,
                      As, Bs);
  }
}

constexpr int kSWarps = 4;

__global__ void __launch_bounds__(kSWarps * 32)
k_project_small(const ProjTask* __restrict__ tasks, int64_t n, const int32_t* __restrict__ D,
                const int32_t* __restrict__ m, const int64_t* __restrict__ uoff,
                const double* __restrict__ X, const double* __restrict__ U,
                double* __restrict__ Y) {
  __shared__ double Ts[kSWarps][kPT][kPS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double (*T)[kPS] = Ts[warp];
  for (int64_t b = int64_t(blockIdx.x) * kSWarps + warp; b < n; b += int64_t(gridDim.x) * kSWarps) {
    const ProjTask pt = tasks[b];
    const int Do = D[pt.so], Di = D[pt.si], mo = m[pt.so], mi = m[pt.si];
    const double* Xb = X + pt.xoff;
    const double* Ui = U + uoff[pt.si];
    const double* Uo = U + uoff[pt.so];
    double* Yb = Y + pt.yoff;
    const int groups = 32 / mi;          // mi <= Di <= 32
    const int cc = lane % mi, g = lane / mi;
    if (g < groups) {
      for (int i = g; i < Do; i += groups) {
        double acc = 0.0;
        for (int k = 0; k < Di; ++k) acc = fma(Xb[i * Di + k], Ui[k * mi + cc], acc);
        T[i][cc] = acc;
      }
    }
    __syncwarp();
    if (g < groups) {
      for (int a = g; a < mo; a += groups) {
        double acc = 0.0;
        for (int i = 0; i < Do; ++i) acc = fma(Uo[i * mo + a], T[i][cc], acc);
        Yb[a * mi + cc] = acc;
      }
    }
    __syncwarp();
  }
}

}  // namespace

void project_small(const ProjTask* tasks, int64_t n, const int32_t* D, const int32_t* m,
                   const int64_t* uoff, const double* X, const double* U, double* Y,
                   cudaStream_t s) {
  if (n <= 0) return;
  const int64_t blocks = std::min<int64_t>((n + kSWarps - 1) / kSWarps, 152 * 16 * 32);
  k_project_small<<<int(blocks), kSWarps * 32, 0, s>>>(tasks, n, D, m, uoff, X, U, Y);
  DMRG_LAUNCHED();
}

void project_blocks(const ProjTask* tasks, const int64_t* tile_beg1, int64_t n_tiles1,
                    const int64_t* tile_beg2, int64_t n_tiles2, int64_t n, const int32_t* D,
                    const int32_t* m, const int64_t* uoff, const double* X, const double* U,
                    double* T, double* Y, cudaStream_t s) {
  if (n <= 0) return;
  const int64_t cap = 152 * 16 * 64;
  if (n_tiles1 > 0) {
    k_project<1><<<int(std::min(n_tiles1, cap)), kPThreads, 0, s>>>(tasks, tile_beg1, n, D, m,
                                                                     uoff, X, U, T, Y);
    DMRG_LAUNCHED();
  }
  if (n_tiles2 > 0) {
    k_project<2><<<int(std::min(n_tiles2, cap)), kPThreads, 0, s>>>(tasks, tile_beg2, n, D, m,
                                                                     uoff, X, U, T, Y);
    DMRG_LAUNCHED();
  }
}

}  // namespace dmrg
