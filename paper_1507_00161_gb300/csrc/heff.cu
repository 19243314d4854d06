// Fused superblock product  psi'(b') = sum_k s_k L_k[Q_L' <- Q_L] psi(b) R_k[Q_R' <- Q_R]^T
// (the two-site H_eff of the superblock "Xi_l (x) Lambda (x) Lambda (x) Xi_r").
//
// Work unit (one thread block, four warps): a group of at most 64 terms of one output
// tile (at most 32 x 32 of a psi' block).  Each warp takes every fourth term of the group.
// Operator blocks and psi blocks start on 16-byte boundaries, so a warp streams the three
// blocks of a term (L rows of the tile, R rows of the tile, psi_in) into a shared-memory
// ring with 16-byte cp.async copies, up to four terms ahead of the one it computes
// (completion in commit-group order; no spin-waits).  Compute from shared memory with a
// fixed lane map: lane = (column c, row group g), rows g, g+G, ... with G = 32 / n:
//     X[i][c] = sum_r psi[i][r] R[c][r]        (X in shared memory)
//     acc[i][c] += s sum_k L[i][k] X[k][c]     (acc in registers)
// Terms whose inner dimensions exceed 32 go through a chunked path that reads global
// memory directly.  The warps' partial tiles are added in a fixed order, and groups of one
// tile are added in group order by k_heff_reduce: the result is deterministic.
#include <stdint.h>

#include <mutex>

#include "common.h"

namespace dmrg {

constexpr int kW = 4;          // warps per block
constexpr int kT = 32;         // output tile edge, small-term inner limit
constexpr int kDepth = 4;      // terms in flight per warp
constexpr int kRingBytes = 12288;
constexpr int kXS = kT * (kT + 1);

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_wait_n(int n) {
  switch (n) {
    case 0: cp_wait<0>(); break;
    case 1: cp_wait<1>(); break;
    case 2: cp_wait<2>(); break;
    default: cp_wait<3>(); break;
  }
}

template <class T>
__device__ __forceinline__ int round_vec(int e) {
  constexpr int v = 16 / int(sizeof(T));
  return (e + v - 1) / v * v;
}

// elements a small term occupies in the ring (three 16-byte aligned pieces)
template <class T>
__device__ __forceinline__ int term_elems(int m, int n, int dLi, int dRi) {
  return round_vec<T>(m * dLi) + round_vec<T>(n * dRi) + round_vec<T>(dLi * dRi);
}

// rows x cols of a row-major source (ld) into dst (leading dimension cols), one
// asynchronous copy per element (chunk rows need not start on 16-byte boundaries)
template <class T>
__device__ __forceinline__ void stage_chunk(T* dst, const T* src, int rows, int cols, int ld,
                                            int lane) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "element size");
  for (int e = lane; e < rows * cols; e += 32) {
    const int r = e / cols, cc = e - r * cols;
    const unsigned sm = static_cast<unsigned>(__cvta_generic_to_shared(dst + e));
    const T* g = src + (int64_t)r * ld + cc;
    if (sizeof(T) == 8)
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sm), "l"(g) : "memory");
    else
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sm), "l"(g) : "memory");
  }
}

template <class T>
__device__ __forceinline__ void stage(T* dst, const T* src, int elems, int lane) {
  const int nv = (elems * int(sizeof(T)) + 15) / 16;
  for (int v = lane; v < nv; v += 32)
    cp_async16(reinterpret_cast<char*>(dst) + 16 * v, reinterpret_cast<const char*>(src) + 16 * v);
}

template <class T>
__global__ void __launch_bounds__(kW * 32, sizeof(T) == 4 ? 4 : 2)
    k_heff_fused(const HeffTile* __restrict__ tiles, const HeffItem* __restrict__ items,
                 const HeffPtrs<T> ptrs) {
  constexpr int kRing = kRingBytes / int(sizeof(T));
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* const base = reinterpret_cast<T*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* const ring = base + warp * (kRing + kXS);
  T* const Xs = ring + kRing;
  __shared__ int slot_pos[kW][kDepth];
  const HeffTile t = tiles[blockIdx.x];
  if (ptrs.active && !ptrs.active[t.inst]) return;   // whole block: uniform
  const T* __restrict__ L = ptrs.L[t.inst];
  const T* __restrict__ R = ptrs.R[t.inst];
  const T* __restrict__ X = ptrs.X[t.inst];
  T* __restrict__ Y = ptrs.Y[t.inst];
  T* __restrict__ P = ptrs.P[t.inst];
  const int m = t.m, n = t.n;
  const int G = 32 / n;                // row groups
  const int c = lane % n, g = lane / n;
  const bool act = g < G;
  const int rows_mine = act ? (m - g + G - 1) / G : 0;   // rows g, g+G, ... < m
  T acc[kT];
#pragma unroll
  for (int q = 0; q < kT; ++q) acc[q] = T(0);

  const int first = t.i0 + warp;
  const int cnt = first < t.i1 ? (t.i1 - first + kW - 1) / kW : 0;
  // ring state: terms in flight occupy [headpos, tail) or, once wrapped,
  // [headpos, end of the used part) and [0, tail)
  int issued = 0, done = 0, inflight = 0, tail = 0, headpos = 0;
  bool wrapped = false;

  while (done < cnt) {
    // prefetch following terms into the ring (circular, in order)
    while (inflight < kDepth && issued < cnt) {
      const HeffItem it = items[first + issued * kW];
      const int S = term_elems<T>(m, n, it.dLi, it.dRi);
      if (it.dLi > kT || it.dRi > kT || S > kRing) break;
      int pos;
      if (inflight == 0) {
        pos = 0;
        wrapped = false;
      } else if (!wrapped) {
        if (tail + S <= kRing) {
          pos = tail;
        } else if (S <= headpos) {
          pos = 0;
          wrapped = true;
        } else {
          break;
        }
      } else {
        if (tail + S <= headpos) pos = tail;
        else break;
      }
      T* dst = ring + pos;
      stage(dst, L + it.loff + (int64_t)t.r0 * it.dLi, m * it.dLi, lane);
      dst += round_vec<T>(m * it.dLi);
      stage(dst, R + it.roff + (int64_t)t.c0 * it.dRi, n * it.dRi, lane);
      dst += round_vec<T>(n * it.dRi);
      stage(dst, X + it.xoff, it.dLi * it.dRi, lane);
      cp_commit();
      if (lane == 0) slot_pos[warp][issued % kDepth] = pos;
      if (inflight == 0) headpos = pos;
      tail = pos + S;
      ++issued;
      ++inflight;
    }
    const HeffItem it = items[first + done * kW];
    const T sg = T(it.sign);
    const int dLi = it.dLi, dRi = it.dRi;
    if (inflight == 0) {
      // large term: chunks staged into the (empty) ring by asynchronous copies; X rows
      // accumulate in shared memory over the chunks of the psi columns (same order of
      // summation as a single pass)
      ++issued;
      constexpr int KC = kRing / (3 * kT) < kT ? kRing / (3 * kT) : kT;   // rows per chunk
      T* const Pc = ring;              // psi chunk (kc x rc), then the L chunk (m x kc)
      T* const Rc = ring + KC * kT;    // R chunk (n x rc)
      for (int k0 = 0; k0 < dLi; k0 += KC) {
        const int kc = min(KC, dLi - k0);
        for (int r0 = 0; r0 < dRi; r0 += kT) {
          const int rc = min(kT, dRi - r0);
          stage_chunk(Pc, X + it.xoff + (int64_t)k0 * dRi + r0, kc, rc, dRi, lane);
          stage_chunk(Rc, R + it.roff + (int64_t)t.c0 * dRi + r0, n, rc, dRi, lane);
          cp_commit();
          cp_wait<0>();
          __syncwarp();
          if (act) {
            const T* rr = Rc + c * rc;
            for (int i = g; i < kc; i += G) {
              const T* pr = Pc + i * rc;
              T s = r0 ? Xs[i * (kT + 1) + c] : T(0);
              for (int r = 0; r < rc; ++r) s = fma(pr[r], rr[r], s);
              Xs[i * (kT + 1) + c] = s;
            }
          }
          __syncwarp();
        }
        stage_chunk(Pc, L + it.loff + (int64_t)t.r0 * dLi + k0, m, kc, dLi, lane);
        cp_commit();
        cp_wait<0>();
        __syncwarp();
        if (act) {
          const T* lr = Pc + g * kc;
          for (int k = 0; k < kc; ++k) {
            const T xv = sg * Xs[k * (kT + 1) + c];
#pragma unroll
            for (int q = 0; q < kT; ++q)
              if (q < rows_mine) acc[q] = fma(lr[q * G * kc + k], xv, acc[q]);
          }
        }
        __syncwarp();
      }
      ++done;
      continue;
    }
    // wait for the oldest term in flight (later groups may still be pending)
    cp_wait_n(inflight - 1);
    __syncwarp();
    const T* Ls = ring + slot_pos[warp][done % kDepth];
    const T* Rs = Ls + round_vec<T>(m * dLi);
    const T* Ps = Rs + round_vec<T>(n * dRi);
    // the cheaper association of L psi R^T for this tile: (psi R^T) first or (L psi) first
    const bool lfirst = int64_t(m) * dRi * (dLi + n) < int64_t(n) * dLi * (dRi + m);
    if (!lfirst) {
      if (act) {
        const T* rr = Rs + c * dRi;
        for (int i = g; i < dLi; i += G) {
          const T* pr = Ps + i * dRi;
          T s = T(0);
          for (int r = 0; r < dRi; ++r) s = fma(pr[r], rr[r], s);
          Xs[i * (kT + 1) + c] = s;
        }
      }
      __syncwarp();
      if (act) {
        const T* lr = Ls + g * dLi;
        for (int k = 0; k < dLi; ++k) {
          const T xv = sg * Xs[k * (kT + 1) + c];
#pragma unroll
          for (int q = 0; q < kT; ++q)
            if (q < rows_mine) acc[q] = fma(lr[q * G * dLi + k], xv, acc[q]);
        }
      }
    } else {
      // Z (m x dRi) = L psi in shared memory, then acc[i][c] += s sum_b Z[i][b] R[c][b]
      for (int e = lane; e < m * dRi; e += 32) {
        const int i = e / dRi, b = e - i * dRi;
        const T* lr = Ls + i * dLi;
        T s = T(0);
        for (int a = 0; a < dLi; ++a) s = fma(lr[a], Ps[a * dRi + b], s);
        Xs[i * (kT + 1) + b] = s;
      }
      __syncwarp();
      if (act) {
        const T* rr = Rs + c * dRi;
        for (int b = 0; b < dRi; ++b) {
          const T rv = sg * rr[b];
#pragma unroll
          for (int q = 0; q < kT; ++q)
            if (q < rows_mine) acc[q] = fma(Xs[(g + q * G) * (kT + 1) + b], rv, acc[q]);
        }
      }
    }
    __syncwarp();
    ++done;
    --inflight;
    if (inflight > 0) {
      const int np = slot_pos[warp][done % kDepth];
      if (np < headpos) wrapped = false;   // the head crossed into the wrapped part
      headpos = np;
    } else {
      tail = headpos = 0;
      wrapped = false;
    }
  }
  cp_wait<0>();
  // fixed-order reduction of the warps' partial tiles (reuses the rings)
  __syncthreads();
  T* const red = base + warp * (kRing + kXS);
  if (act) {
#pragma unroll
    for (int q = 0; q < kT; ++q)
      if (q < rows_mine) red[(g + q * G) * n + c] = acc[q];
  }
  __syncthreads();
  const int mn = m * n;
  for (int e = threadIdx.x; e < mn; e += kW * 32) {
    T s = base[e];
#pragma unroll
    for (int w = 1; w < kW; ++w) s += base[w * (kRing + kXS) + e];
    if (t.poff < 0) {
      const int i = e / n, cc = e - i * n;
      Y[t.yoff + (int64_t)(t.r0 + i) * t.ld + t.c0 + cc] = s;
    } else {
      P[t.poff + e] = s;
    }
  }
}

// psi' tile = sum over groups (in group order) of the partial tiles
template <class T>
__global__ void k_heff_reduce(const HeffRed* __restrict__ red, const HeffPtrs<T> ptrs) {
  const HeffRed r = red[blockIdx.x];
  if (ptrs.active && !ptrs.active[r.inst]) return;
  const T* __restrict__ P = ptrs.P[r.inst];
  T* __restrict__ Y = ptrs.Y[r.inst];
  const int mn = r.m * r.n;
  for (int e = threadIdx.x; e < mn; e += blockDim.x) {
    T s = T(0);
    for (int g = 0; g < r.groups; ++g) s += P[r.poff + (int64_t)g * mn + e];
    const int i = e / r.n, c = e - i * r.n;
    Y[r.yoff + (int64_t)(r.r0 + i) * r.ld + r.c0 + c] = s;
  }
}

// psi blocks into a 16-byte aligned copy (optionally converted): one block per thread block
template <class TI, class TO>
__global__ void k_pad_psi(const TI* __restrict__ x, TO* __restrict__ xp,
                          const int64_t* __restrict__ src_off, const int64_t* __restrict__ dst_off,
                          const int32_t* __restrict__ len) {
  const int b = blockIdx.x;
  const TI* s = x + src_off[b];
  TO* d = xp + dst_off[b];
  for (int i = threadIdx.x; i < len[b]; i += blockDim.x) d[i] = TO(s[i]);
}

template <class T>
void heff_reduce(const HeffRed* d_red, int64_t n_red, const HeffPtrs<T>& ptrs, cudaStream_t s) {
  if (n_red <= 0) return;
  k_heff_reduce<T><<<int(n_red), 128, 0, s>>>(d_red, ptrs);
  DMRG_LAUNCHED();
}
template void heff_reduce<float>(const HeffRed*, int64_t, const HeffPtrs<float>&, cudaStream_t);
template void heff_reduce<double>(const HeffRed*, int64_t, const HeffPtrs<double>&, cudaStream_t);

template <class T>
void heff_fused(const HeffTile* d_tiles, int64_t n_tiles, const HeffItem* d_items,
                const HeffRed* d_red, int64_t n_red, const HeffPtrs<T>& ptrs, cudaStream_t s) {
  if (n_tiles > 0) {
    const size_t smem = sizeof(T) * kW * (kRingBytes / sizeof(T) + kXS);
    static std::once_flag attr_once;   // per process: the attribute belongs to the kernel
    std::call_once(attr_once, [&] {
      DMRG_CUDA(cudaFuncSetAttribute(k_heff_fused<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(smem)));
    });
    k_heff_fused<T><<<int(n_tiles), kW * 32, smem, s>>>(d_tiles, d_items, ptrs);
    DMRG_LAUNCHED();
  }
  heff_reduce<T>(d_red, n_red, ptrs, s);   // partial tiles of both product kernels
}
template void heff_fused<double>(const HeffTile*, int64_t, const HeffItem*, const HeffRed*,
                                 int64_t, const HeffPtrs<double>&, cudaStream_t);

// staging with the vector pointer read from device memory (graph replay on new vectors)
template <class TO>
__global__ void k_pad_psi_ind(const double* const* __restrict__ xptr, TO* __restrict__ xp,
                              const int64_t* __restrict__ src_off,
                              const int64_t* __restrict__ dst_off,
                              const int32_t* __restrict__ len, const int32_t* __restrict__ active) {
  if (active && !active[0]) return;
  const int b = blockIdx.x;
  const double* s = xptr[0] + src_off[b];
  TO* d = xp + dst_off[b];
  for (int i = threadIdx.x; i < len[b]; i += blockDim.x) d[i] = TO(s[i]);
}

template <class TI>
__global__ void k_out_to_f64_ind(const TI* __restrict__ y, double* const* __restrict__ optr,
                                 int64_t n, const int32_t* __restrict__ active) {
  if (active && !active[0]) return;
  double* o = optr[0];
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    o[i] = double(y[i]);
}

template <class TO>
void pad_psi_ind(const double* const* x_ptr, TO* xp, const int64_t* src_off,
                 const int64_t* dst_off, const int32_t* len, int nblocks, const int32_t* active,
                 cudaStream_t s) {
  if (nblocks <= 0) return;
  k_pad_psi_ind<TO><<<nblocks, 128, 0, s>>>(x_ptr, xp, src_off, dst_off, len, active);
  DMRG_LAUNCHED();
}
template void pad_psi_ind<float>(const double* const*, float*, const int64_t*, const int64_t*,
                                 const int32_t*, int, const int32_t*, cudaStream_t);
template void pad_psi_ind<double>(const double* const*, double*, const int64_t*, const int64_t*,
                                  const int32_t*, int, const int32_t*, cudaStream_t);

template <class TI>
void out_to_f64_ind(const TI* y, double* const* out_ptr, int64_t n, const int32_t* active,
                    cudaStream_t s) {
  if (n <= 0) return;
  const int blocks = int(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)));
  k_out_to_f64_ind<TI><<<blocks, 256, 0, s>>>(y, out_ptr, n, active);
  DMRG_LAUNCHED();
}
template void out_to_f64_ind<float>(const float*, double* const*, int64_t, const int32_t*,
                                    cudaStream_t);
template void out_to_f64_ind<double>(const double*, double* const*, int64_t, const int32_t*,
                                     cudaStream_t);

template <class TO>
void pad_psi(const double* x, TO* xp, const int64_t* src_off, const int64_t* dst_off,
             const int32_t* len, int nblocks, cudaStream_t s) {
  if (nblocks <= 0) return;
  k_pad_psi<double, TO><<<nblocks, 128, 0, s>>>(x, xp, src_off, dst_off, len);
  DMRG_LAUNCHED();
}
template void pad_psi<double>(const double*, double*, const int64_t*, const int64_t*,
                              const int32_t*, int, cudaStream_t);
template void pad_psi<float>(const double*, float*, const int64_t*, const int64_t*,
                             const int32_t*, int, cudaStream_t);

}  // namespace dmrg
