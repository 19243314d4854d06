// Fused superblock product  psi'(b') = sum_k s_k L_k[Q_L' <- Q_L] psi(b) R_k[Q_R' <- Q_R]^T
// (the two-site H_eff of the superblock "Xi_l (x) Lambda (x) Lambda (x) Xi_r").
//
// One thread block per group of at most 64 terms of an output tile (at most 32 x 32 of a
// psi' block), four warps splitting the group's terms; tiles with more terms write partial
// tiles that a second kernel adds in group order.  Per term a warp stages the operator blocks it needs in shared memory
// (16-byte vector loads when a block is contiguous: block offsets are 16-byte aligned),
// forms X = psi_in R^T in shared memory (lanes over X elements), and accumulates s L X
// into registers (lanes over output elements, so small blocks keep the lanes busy).
// Inner dimensions are processed in chunks of 16.  The warps' partial tiles are added in a
// fixed order: deterministic, no atomics.  Every
// operator block is read once per product (outputs wider than one tile re-read the rows
// they need), so the product is bound by HBM bandwidth.
#include <stdint.h>

#include "common.h"

namespace dmrg {

constexpr int kC = 32;   // output tile edge
constexpr int kK = 16;   // inner chunk
constexpr int kW = 4;    // warps per block
constexpr int kLS = kC * kK + 8;
constexpr int kRS = kC * kK + 8;
constexpr int kXS = kK * kC + 8;
constexpr int kPerWarp = kLS + kRS + kXS;   // >= kC * kC: reused for the reduction

template <class T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
  static constexpr int n = 4;
};
template <>
struct Vec16<double> {
  using type = double2;
  static constexpr int n = 2;
};

// rows x cols of a row-major source (leading dimension ld) into dst (leading dimension
// cols); 16-byte vectors when the region is contiguous and aligned (may write up to one
// vector past rows*cols: the buffers are padded)
template <class T>
__device__ __forceinline__ void warp_stage(T* __restrict__ dst, const T* __restrict__ src, int rows,
                                           int cols, int ld, int lane) {
  using V = typename Vec16<T>::type;
  constexpr int VN = Vec16<T>::n;
  const int tot = rows * cols;
  if (cols == ld && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
    const int nv = (tot + VN - 1) / VN;
    const V* s = reinterpret_cast<const V*>(src);
    V* d = reinterpret_cast<V*>(dst);
    for (int v = lane; v < nv; v += 32) d[v] = __ldg(s + v);
  } else {
    for (int e = lane; e < tot; e += 32) {
      const int r = e / cols, c = e - r * cols;
      dst[e] = __ldg(src + (int64_t)r * ld + c);
    }
  }
}

template <class T>
__global__ void __launch_bounds__(kW * 32, sizeof(T) == 4 ? 6 : 3) k_heff_fused(const HeffTile* __restrict__ tiles,
                                                           const HeffItem* __restrict__ items,
                                                           const T* __restrict__ L,
                                                           const T* __restrict__ R,
                                                           const T* __restrict__ X,
                                                           T* __restrict__ Y,
                                                           T* __restrict__ P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* const base = reinterpret_cast<T*>(smem_raw);
  const HeffTile t = tiles[blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* const Ls = base + warp * kPerWarp;
  T* const Rs = Ls + kLS;
  T* const Xs = Rs + kRS;
  const int m = t.m, n = t.n, mn = m * n;
  T acc[kC];
#pragma unroll
  for (int q = 0; q < kC; ++q) acc[q] = T(0);
  for (int j = t.i0 + warp; j < t.i1; j += kW) {
    const HeffItem it = items[j];
    const int dLi = it.dLi, dRi = it.dRi;
    const T sg = T(it.sign);
    for (int k0 = 0; k0 < dLi; k0 += kK) {
      const int kc = min(kK, dLi - k0);
      // X (kc x n) = psi_in[k0.., :] R[c0.., :]^T, inner dimension in chunks
      for (int e = lane; e < kc * n; e += 32) Xs[e] = T(0);
      for (int r0 = 0; r0 < dRi; r0 += kK) {
        const int rc = min(kK, dRi - r0);
        warp_stage(Rs, R + it.roff + (int64_t)t.c0 * dRi + r0, n, rc, dRi, lane);
        __syncwarp();
        const T* __restrict__ P = X + it.xoff + (int64_t)k0 * dRi + r0;
        for (int e = lane; e < kc * n; e += 32) {
          const int i = e / n, c = e - i * n;
          const T* pr = P + (int64_t)i * dRi;
          const T* rr = Rs + c * rc;
          T s = T(0);
          for (int r = 0; r < rc; ++r) s = fma(__ldg(pr + r), rr[r], s);
          Xs[e] += s;
        }
        __syncwarp();
      }
      warp_stage(Ls, L + it.loff + (int64_t)t.r0 * dLi + k0, m, kc, dLi, lane);
      __syncwarp();
#pragma unroll
      for (int q = 0; q < kC; ++q) {
        const int e = lane + 32 * q;
        if (e < mn) {
          const int i = e / n, c = e - i * n;
          const T* lr = Ls + i * kc;
          const T* xc = Xs + c;
          T s = T(0);
          for (int k = 0; k < kc; ++k) s = fma(lr[k], xc[k * n], s);
          acc[q] = fma(sg, s, acc[q]);
        }
      }
      __syncwarp();
    }
  }
  // fixed-order reduction of the warps' partial tiles
  __syncthreads();
  T* const red = base + warp * kPerWarp;
#pragma unroll
  for (int q = 0; q < kC; ++q) {
    const int e = lane + 32 * q;
    if (e < mn) red[e] = acc[q];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < mn; e += kW * 32) {
    const int i = e / n, c = e - i * n;
    T s = base[e];
#pragma unroll
    for (int w = 1; w < kW; ++w) s += base[w * kPerWarp + e];
    if (t.poff < 0) Y[t.yoff + (int64_t)(t.r0 + i) * t.ld + t.c0 + c] = s;
    else P[t.poff + e] = s;
  }
}

// psi' tile = sum over groups (in group order) of the partial tiles
template <class T>
__global__ void k_heff_reduce(const HeffRed* __restrict__ red, const T* __restrict__ P,
                              T* __restrict__ Y) {
  const HeffRed r = red[blockIdx.x];
  const int mn = r.m * r.n;
  for (int e = threadIdx.x; e < mn; e += blockDim.x) {
    T s = T(0);
    for (int g = 0; g < r.groups; ++g) s += P[r.poff + (int64_t)g * mn + e];
    const int i = e / r.n, c = e - i * r.n;
    Y[r.yoff + (int64_t)(r.r0 + i) * r.ld + r.c0 + c] = s;
  }
}

template <class T>
void heff_fused(const HeffTile* d_tiles, int64_t n_tiles, const HeffItem* d_items,
                const HeffRed* d_red, int64_t n_red, const T* L, const T* R, const T* X, T* Y,
                T* partial, cudaStream_t s) {
  if (n_tiles <= 0) return;
  const size_t smem = sizeof(T) * kW * kPerWarp;
  static bool attr_set = false;   // per process: the attribute belongs to the kernel
  if (!attr_set) {
    DMRG_CUDA(cudaFuncSetAttribute(k_heff_fused<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   int(smem)));
    attr_set = true;
  }
  k_heff_fused<T><<<int(n_tiles), kW * 32, smem, s>>>(d_tiles, d_items, L, R, X, Y, partial);
  DMRG_LAUNCHED();
  if (n_red > 0) {
    k_heff_reduce<T><<<int(n_red), 128, 0, s>>>(d_red, partial, Y);
    DMRG_LAUNCHED();
  }
}
template void heff_fused<double>(const HeffTile*, int64_t, const HeffItem*, const HeffRed*,
                                 int64_t, const double*, const double*, const double*, double*,
                                 double*, cudaStream_t);
template void heff_fused<float>(const HeffTile*, int64_t, const HeffItem*, const HeffRed*,
                                int64_t, const float*, const float*, const float*, float*,
                                float*, cudaStream_t);

}  // namespace dmrg
