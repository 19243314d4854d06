// Fused superblock product on the tensor cores (mixed path: FP32 storage, FP32 accumulate)
//     psi'(b') = sum_k s_k L_k[Q_L' <- Q_L] psi(b) R_k[Q_R' <- Q_R]^T
//
// Same work decomposition and shared-memory ring as the FP64 kernel in heff.cu (a thread
// block = a group of at most 64 terms of a 32 x 32 output tile, four warps, cp.async
// prefetch of up to four terms per warp), but both small products of a term run as warp
// matrix multiply-accumulates m16n8k8 on TF32 operands split into high and low parts:
//     a b  ~  a_hi b_hi + a_hi b_lo + a_lo b_hi   (three MMAs, FP32 accumulation)
// which keeps FP32-level accuracy (the dropped a_lo b_lo term is ~2^-22 relative).  This
// kernel takes the output blocks up to the big-block edge (dmrg_set_tuning): in the first
// sweeps from a random start they are a few states wide, well below the 64-row minimum of
// a CTA-level MMA, so the warp-level instruction is the one that fits them; wider blocks
// (hundreds of states in converged sweeps at M = 4096) go to the grouped GEMM passes of
// tgemm.cu.
//     X (dLi x n)  = psi (dLi x dRi) R^T        (M = dLi, N = n, K = dRi)
//     Y (m x n)   += s L (m x dLi) X             (M = m,   N = n, K = dLi)
// Terms with an inner dimension above 32 are processed in 32-wide chunks staged by
// asynchronous copies (the L chunk in flight while the psi and R chunks load).
// Deterministic: fixed term order per warp, fixed warp and group order.
#include <stdint.h>

#include <mutex>

#include "common.h"

namespace dmrg {
namespace tc {

constexpr int kW = 4;
constexpr int kT = 32;
constexpr int kDepth = 4;
constexpr int kRing = 12288 / 4;    // floats per warp ring
constexpr int kXLD = 36;            // leading dimension of X in shared memory
constexpr int kXS = kT * kXLD;

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
__device__ __forceinline__ int rv(int e) { return (e + 3) & ~3; }   // 16-byte rounding

__device__ __forceinline__ void stage_async(float* dst, const float* src, int elems, int lane) {
  const int nv = (elems + 3) >> 2;
  for (int v = lane; v < nv; v += 32) cp_async16(dst + 4 * v, src + 4 * v);
}
// rows x cols of a row-major source (ld) into dst with leading dimension cols, as 4-byte
// asynchronous copies (rows of a chunk need not start on 16-byte boundaries)
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void stage_chunk(float* dst, const float* src, int rows, int cols,
                                            int ld, int lane) {
  for (int e = lane; e < rows * cols; e += 32) {
    const int r = e / cols, c = e - r * cols;
    cp_async4(dst + e, src + (int64_t)r * ld + c);
  }
}

__device__ __forceinline__ uint32_t tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void split(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32(x);
  lo = tf32(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                    uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
// d += a b with operands split into TF32 high and low parts (small products first)
__device__ __forceinline__ void mma3(float (&d)[4], const float (&a)[4], const float (&b)[2]) {
  uint32_t ah[4], al[4], bh[2], bl[2];
#pragma unroll
  for (int i = 0; i < 4; ++i) split(a[i], ah[i], al[i]);
#pragma unroll
  for (int i = 0; i < 2; ++i) split(b[i], bh[i], bl[i]);
  mma(d, al[0], al[1], al[2], al[3], bh[0], bh[1]);
  mma(d, ah[0], ah[1], ah[2], ah[3], bl[0], bl[1]);
  mma(d, ah[0], ah[1], ah[2], ah[3], bh[0], bh[1]);
}

// the same for two accumulators sharing a: their MMA chains are interleaved so that each
// MMA does not wait on the one just issued (same order of the three terms per accumulator)
__device__ __forceinline__ void mma3_2b(float (&d0)[4], float (&d1)[4], const float (&a)[4],
                                        const float (&b0)[2], const float (&b1)[2]) {
  uint32_t ah[4], al[4], bh0[2], bl0[2], bh1[2], bl1[2];
#pragma unroll
  for (int i = 0; i < 4; ++i) split(a[i], ah[i], al[i]);
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    split(b0[i], bh0[i], bl0[i]);
    split(b1[i], bh1[i], bl1[i]);
  }
  mma(d0, al[0], al[1], al[2], al[3], bh0[0], bh0[1]);
  mma(d1, al[0], al[1], al[2], al[3], bh1[0], bh1[1]);
  mma(d0, ah[0], ah[1], ah[2], ah[3], bl0[0], bl0[1]);
  mma(d1, ah[0], ah[1], ah[2], ah[3], bl1[0], bl1[1]);
  mma(d0, ah[0], ah[1], ah[2], ah[3], bh0[0], bh0[1]);
  mma(d1, ah[0], ah[1], ah[2], ah[3], bh1[0], bh1[1]);
}

// element (r, c) of a row-major rows x cols matrix, zero outside
__device__ __forceinline__ float at(const float* M, int ld, int rows, int cols, int r, int c) {
  return (r < rows && c < cols) ? M[r * ld + c] : 0.f;
}

// cX[mt][nt] += P (rows x kdim, ld ldp) * R^T, R is n x kdim (ld ldr)
__device__ __forceinline__ void stage1(float (&cX)[2][4][4], const float* P, int ldp, int rows,
                                       const float* R, int ldr, int n, int kdim, int MT, int NT,
                                       int gid, int tig) {
  const int KS = (kdim + 7) >> 3;
  for (int ks = 0; ks < KS; ++ks) {
    const int k0 = ks * 8 + tig, k1 = k0 + 4;
#pragma unroll
    for (int nt = 0; nt < 4; nt += 2) {   // column tiles in pairs (interleaved chains)
      if (nt >= NT) break;
      const int col = nt * 8 + gid;
      const float b[2] = {at(R, ldr, n, kdim, col, k0), at(R, ldr, n, kdim, col, k1)};
      const bool two = nt + 1 < NT;
      const float b1[2] = {two ? at(R, ldr, n, kdim, col + 8, k0) : 0.f,
                           two ? at(R, ldr, n, kdim, col + 8, k1) : 0.f};
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        if (mt >= MT) break;
        const int r0 = mt * 16 + gid, r1 = r0 + 8;
        const float a[4] = {at(P, ldp, rows, kdim, r0, k0), at(P, ldp, rows, kdim, r1, k0),
                            at(P, ldp, rows, kdim, r0, k1), at(P, ldp, rows, kdim, r1, k1)};
        if (two) mma3_2b(cX[mt][nt], cX[mt][nt + 1], a, b, b1);
        else mma3(cX[mt][nt], a, b);
      }
    }
  }
}

// X (shared, kXLD) = s cX ; padding rows / columns come out zero (zero operands)
__device__ __forceinline__ void store_x(float* Xs, const float (&cX)[2][4][4], float s, int MT,
                                        int NT, int gid, int tig) {
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    if (mt >= MT) break;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      if (nt >= NT) break;
      const int r = mt * 16 + gid, c = nt * 8 + 2 * tig;
      Xs[r * kXLD + c] = s * cX[mt][nt][0];
      Xs[r * kXLD + c + 1] = s * cX[mt][nt][1];
      Xs[(r + 8) * kXLD + c] = s * cX[mt][nt][2];
      Xs[(r + 8) * kXLD + c + 1] = s * cX[mt][nt][3];
    }
  }
}

// acc[mt][nt] += L (m x kdim, ld ldl) * X (kdim x n, shared)
__device__ __forceinline__ void stage2(float (&acc)[2][4][4], const float* Ls, int ldl, int m,
                                       int kdim, const float* Xs, int MT, int NT, int gid,
                                       int tig) {
  const int KS = (kdim + 7) >> 3;
  for (int ks = 0; ks < KS; ++ks) {
    const int k0 = ks * 8 + tig, k1 = k0 + 4;
#pragma unroll
    for (int nt = 0; nt < 4; nt += 2) {   // column tiles in pairs (interleaved chains)
      if (nt >= NT) break;
      const int col = nt * 8 + gid;
      const float b[2] = {Xs[k0 * kXLD + col], Xs[k1 * kXLD + col]};
      const bool two = nt + 1 < NT;
      const float b1[2] = {Xs[k0 * kXLD + col + 8], Xs[k1 * kXLD + col + 8]};
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        if (mt >= MT) break;
        const int r0 = mt * 16 + gid, r1 = r0 + 8;
        const float a[4] = {at(Ls, ldl, m, kdim, r0, k0), at(Ls, ldl, m, kdim, r1, k0),
                            at(Ls, ldl, m, kdim, r0, k1), at(Ls, ldl, m, kdim, r1, k1)};
        if (two) mma3_2b(acc[mt][nt], acc[mt][nt + 1], a, b, b1);
        else mma3(acc[mt][nt], a, b);
      }
    }
  }
}

__global__ void __launch_bounds__(kW * 32, 3)
    k_heff_tc(const HeffTile* __restrict__ tiles, const HeffItem* __restrict__ items,
              const HeffPtrs<float> ptrs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* const base = reinterpret_cast<float*>(smem_raw);
  __shared__ int slot_pos[kW][kDepth];
  const HeffTile t = tiles[blockIdx.x];
  if (ptrs.active && !ptrs.active[t.inst]) return;   // whole block: uniform
  const float* __restrict__ L = ptrs.L[t.inst];
  const float* __restrict__ R = ptrs.R[t.inst];
  const float* __restrict__ X = ptrs.X[t.inst];
  float* __restrict__ Y = ptrs.Y[t.inst];
  float* __restrict__ P = ptrs.P[t.inst];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gid = lane >> 2, tig = lane & 3;
  float* const ring = base + warp * (kRing + kXS);
  float* const Xs = ring + kRing;
  const int m = t.m, n = t.n;
  const int NT = (n + 7) >> 3, MT2 = (m + 15) >> 4;
  float acc[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[a][b][e] = 0.f;

  const int first = t.i0 + warp;
  const int cnt = first < t.i1 ? (t.i1 - first + kW - 1) / kW : 0;
  int issued = 0, done = 0, inflight = 0, tail = 0, headpos = 0;
  bool wrapped = false;

  while (done < cnt) {
    while (inflight < kDepth && issued < cnt) {
      const HeffItem it = items[first + issued * kW];
      const int S = rv(m * it.dLi) + rv(n * it.dRi) + rv(it.dLi * it.dRi);
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
      float* dst = ring + pos;
      stage_async(dst, L + it.loff + (int64_t)t.r0 * it.dLi, m * it.dLi, lane);
      dst += rv(m * it.dLi);
      stage_async(dst, R + it.roff + (int64_t)t.c0 * it.dRi, n * it.dRi, lane);
      dst += rv(n * it.dRi);
      stage_async(dst, X + it.xoff, it.dLi * it.dRi, lane);
      cp_commit();
      if (lane == 0) slot_pos[warp][issued % kDepth] = pos;
      if (inflight == 0) headpos = pos;
      tail = pos + S;
      ++issued;
      ++inflight;
    }
    const HeffItem it = items[first + done * kW];
    const int dLi = it.dLi, dRi = it.dRi;
    if (inflight == 0) {
      // large term: 32-wide chunks staged synchronously into the (empty) ring
      ++issued;
      // (asynchronous copies: the L chunk is in flight while the psi and R chunks load)
      float* const Pc = ring;                 // psi chunk (kc x rc)
      float* const Rc = ring + kT * kT;       // R chunk (n x rc)
      float* const Lc = ring + 2 * kT * kT;   // L chunk (m x kc)
      for (int k0 = 0; k0 < dLi; k0 += kT) {
        const int kc = min(kT, dLi - k0);
        const int MT1 = (kc + 15) >> 4;
        stage_chunk(Lc, L + it.loff + (int64_t)t.r0 * dLi + k0, m, kc, dLi, lane);
        cp_commit();
        float cX[2][4][4];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int e = 0; e < 4; ++e) cX[a][b][e] = 0.f;
        for (int r0 = 0; r0 < dRi; r0 += kT) {
          const int rc = min(kT, dRi - r0);
          stage_chunk(Pc, X + it.xoff + (int64_t)k0 * dRi + r0, kc, rc, dRi, lane);
          stage_chunk(Rc, R + it.roff + (int64_t)t.c0 * dRi + r0, n, rc, dRi, lane);
          cp_commit();
          cp_wait<0>();
          __syncwarp();
          stage1(cX, Pc, rc, kc, Rc, rc, n, rc, MT1, NT, gid, tig);
          __syncwarp();
        }
        store_x(Xs, cX, it.sign, MT1, NT, gid, tig);
        __syncwarp();
        stage2(acc, Lc, kc, m, kc, Xs, MT2, NT, gid, tig);
        __syncwarp();
      }
      ++done;
      continue;
    }
    cp_wait_n(inflight - 1);
    __syncwarp();
    const float* Ls = ring + slot_pos[warp][done % kDepth];
    const float* Rs = Ls + rv(m * dLi);
    const float* Ps = Rs + rv(n * dRi);
    {
      const int MT1 = (dLi + 15) >> 4;
      float cX[2][4][4];
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
          for (int e = 0; e < 4; ++e) cX[a][b][e] = 0.f;
      stage1(cX, Ps, dRi, dLi, Rs, dRi, n, dRi, MT1, NT, gid, tig);
      store_x(Xs, cX, it.sign, MT1, NT, gid, tig);
    }
    __syncwarp();
    stage2(acc, Ls, dLi, m, dLi, Xs, MT2, NT, gid, tig);
    __syncwarp();
    ++done;
    --inflight;
    if (inflight > 0) {
      const int np = slot_pos[warp][done % kDepth];
      if (np < headpos) wrapped = false;
      headpos = np;
    } else {
      tail = headpos = 0;
      wrapped = false;
    }
  }
  cp_wait<0>();
  // fixed-order reduction of the warps' partial tiles (reuses the rings)
  __syncthreads();
  float* const red = base + warp * (kRing + kXS);
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    if (mt >= MT2) break;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      if (nt >= NT) break;
      const int r = mt * 16 + gid, c = nt * 8 + 2 * tig;
      if (r < m && c < n) red[r * n + c] = acc[mt][nt][0];
      if (r < m && c + 1 < n) red[r * n + c + 1] = acc[mt][nt][1];
      if (r + 8 < m && c < n) red[(r + 8) * n + c] = acc[mt][nt][2];
      if (r + 8 < m && c + 1 < n) red[(r + 8) * n + c + 1] = acc[mt][nt][3];
    }
  }
  __syncthreads();
  const int mn = m * n;
  for (int e = threadIdx.x; e < mn; e += kW * 32) {
    float s = base[e];
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

}  // namespace tc

void heff_tc(const HeffTile* d_tiles, int64_t n_tiles, const HeffItem* d_items,
             const HeffRed* d_red, int64_t n_red, const HeffPtrs<float>& ptrs, cudaStream_t s) {
  if (n_tiles > 0) {
    const size_t smem = sizeof(float) * tc::kW * (tc::kRing + tc::kXS);
    static std::once_flag attr_once;   // per process: the attribute belongs to the kernel
    std::call_once(attr_once, [&] {
      DMRG_CUDA(cudaFuncSetAttribute(tc::k_heff_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(smem)));
    });
    tc::k_heff_tc<<<int(n_tiles), tc::kW * 32, smem, s>>>(d_tiles, d_items, ptrs);
    DMRG_LAUNCHED();
  }
  heff_reduce<float>(d_red, n_red, ptrs, s);   // partial tiles of both product kernels
}

}  // namespace dmrg
