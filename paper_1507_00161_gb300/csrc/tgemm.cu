// Grouped GEMM on the tensor cores for the large sector blocks of the mixed path:
//     C (M x N) (+)= sum_t alpha_t op(A_t) op(B_t)
// over the task lists of kernels.cu (GemmTask / GemmTerm, 64 x 64 output tiles), with
// operands read from FP64 or FP32 arrays.  Each operand element is converted to FP32 and
// split into TF32 high and low parts while it is staged into shared memory; a product is
// three warp MMAs m16n8k8 (lo.hi + hi.lo + hi.hi) with FP32 accumulation (the dropped
// lo.lo term is ~2^-22 relative).  The tensor cores' FP32 accumulation is coarser than
// round-to-nearest (measured: ~7e-6 relative after K = 1000 products), and a stage-2 task
// of the superblock product sums thousands of products, so every 32-wide K chunk starts a
// fresh MMA accumulator and the chunk results are added with compensated (Kahan)
// summation in FP32.  C is written as FP32 or FP64.
//
// Thread block: 128 threads, 2 x 2 warps of 32 x 32 outputs (2 x 4 MMA tiles each); the K
// dimension of every term runs in chunks of 32.  The next chunk is loaded from global
// memory into registers while the tensor cores work on the current one from shared memory.
// Deterministic: fixed term and chunk order, no atomics.
#include <stdint.h>

#include "common.h"

namespace dmrg {

namespace {

constexpr int kTM = 64, kTN = 64, kTK = 32, kThreads = 128;
constexpr int kALd = kTK + 4;    // A tile row (m) stride in words: conflict-free fragments
constexpr int kBLd = kTN + 8;    // B tile row (k) stride in words

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4],
                                         const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <class T>
__device__ __forceinline__ float ld_elem(const T* p) {
  return float(__ldg(p));
}

// one chunk of the flattened (term, k0) sequence of a task, held in registers
struct Chunk {
  float a[kTM * kTK / kThreads];   // 16 elements of A
  float b[kTK * kTN / kThreads];   // 16 elements of B
};

template <class TA, class TB>
__device__ __forceinline__ void load_chunk(Chunk& ch, const GemmTerm& g, const TA* A,
                                           const TB* B, int m0, int n0, int M, int N, int k0,
                                           int tid) {
  const int ta = g.trans & 1, tb = (g.trans >> 1) & 1;
  const float alpha = float(g.alpha);
  const int kr = g.K - k0;
#pragma unroll
  for (int i = 0; i < kTM * kTK / kThreads; ++i) {
    const int idx = tid + kThreads * i;
    int m, k;
    if (!ta) {   // A row-major M x K: k fastest
      m = idx / kTK;
      k = idx - m * kTK;
    } else {     // A stored K x M: m fastest
      k = idx / kTM;
      m = idx - k * kTM;
    }
    float v = 0.f;
    if (m0 + m < M && k < kr)
      v = alpha * ld_elem(ta ? A + int64_t(k0 + k) * g.A.ld + m0 + m
                             : A + int64_t(m0 + m) * g.A.ld + k0 + k);
    ch.a[i] = v;
  }
#pragma unroll
  for (int i = 0; i < kTK * kTN / kThreads; ++i) {
    const int idx = tid + kThreads * i;
    int k, n;
    if (!tb) {   // B row-major K x N: n fastest
      k = idx / kTN;
      n = idx - k * kTN;
    } else {     // B stored N x K: k fastest
      n = idx / kTK;
      k = idx - n * kTK;
    }
    float v = 0.f;
    if (n0 + n < N && k < kr)
      v = ld_elem(tb ? B + int64_t(n0 + n) * g.B.ld + k0 + k : B + int64_t(k0 + k) * g.B.ld + n0 + n);
    ch.b[i] = v;
  }
}

__device__ __forceinline__ void store_chunk(const Chunk& ch, int ta, int tb, uint32_t* Ah,
                                            uint32_t* Al, uint32_t* Bh, uint32_t* Bl,
                                            int tid) {
#pragma unroll
  for (int i = 0; i < kTM * kTK / kThreads; ++i) {
    const int idx = tid + kThreads * i;
    int m, k;
    if (!ta) {
      m = idx / kTK;
      k = idx - m * kTK;
    } else {
      k = idx / kTM;
      m = idx - k * kTM;
    }
    const uint32_t h = to_tf32(ch.a[i]);
    Ah[m * kALd + k] = h;
    Al[m * kALd + k] = to_tf32(ch.a[i] - __uint_as_float(h));
  }
#pragma unroll
  for (int i = 0; i < kTK * kTN / kThreads; ++i) {
    const int idx = tid + kThreads * i;
    int k, n;
    if (!tb) {
      k = idx / kTN;
      n = idx - k * kTN;
    } else {
      n = idx / kTK;
      k = idx - n * kTK;
    }
    const uint32_t h = to_tf32(ch.b[i]);
    Bh[k * kBLd + n] = h;
    Bl[k * kBLd + n] = to_tf32(ch.b[i] - __uint_as_float(h));
  }
}

template <class TA, class TB, class TC>
__global__ void __launch_bounds__(kThreads, 3)
    k_gemm_tc(const GemmTile* __restrict__ tiles, const GemmTask* __restrict__ tasks,
              const GemmTerm* __restrict__ terms, Bases<void> b, int beta_zero,
              const int32_t* __restrict__ active) {
  if (active && !active[0]) return;   // whole block: uniform
  __shared__ __align__(16) uint32_t Ah[kTM * kALd], Al[kTM * kALd];
  __shared__ __align__(16) uint32_t Bh[kTK * kBLd], Bl[kTK * kBLd];
  const GemmTile tl = tiles[blockIdx.x];
  const GemmTask t = tasks[tl.task];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gid = lane >> 2, tig = lane & 3;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  float acc[2][4][4], cmp[2][4][4];   // Kahan sum of the chunk results and its compensation
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][j][e] = cmp[i][j][e] = 0.f;

  // flattened chunk sequence: terms t0..t1, k0 = 0, 32, ... < K
  int jt = t.t0, k0 = 0;
  while (jt < t.t1 && terms[jt].K <= 0) ++jt;
  Chunk ch;
  GemmTerm g{};
  if (jt < t.t1) {
    g = terms[jt];
    load_chunk<TA, TB>(ch, g, static_cast<const TA*>(b.p[g.A.base]) + g.A.off,
                       static_cast<const TB*>(b.p[g.B.base]) + g.B.off, tl.m0, tl.n0, t.M, t.N,
                       k0, tid);
  }
  while (jt < t.t1) {
    store_chunk(ch, g.trans & 1, (g.trans >> 1) & 1, Ah, Al, Bh, Bl, tid);
    __syncthreads();
    // next chunk into registers while this one is multiplied
    int njt = jt, nk0 = k0 + kTK;
    if (nk0 >= g.K) {
      nk0 = 0;
      ++njt;
      while (njt < t.t1 && terms[njt].K <= 0) ++njt;
    }
    GemmTerm ng = g;
    if (njt < t.t1) {
      if (njt != jt) ng = terms[njt];
      load_chunk<TA, TB>(ch, ng, static_cast<const TA*>(b.p[ng.A.base]) + ng.A.off,
                         static_cast<const TB*>(b.p[ng.B.base]) + ng.B.off, tl.m0, tl.n0, t.M,
                         t.N, nk0, tid);
    }
    float part[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) part[i][j][e] = 0.f;
#pragma unroll
    for (int ks = 0; ks < kTK; ks += 8) {
      uint32_t ah[2][4], al[2][4], bh[4][2], bl[4][2];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const int r = wm + mt * 16 + gid;
        ah[mt][0] = Ah[r * kALd + ks + tig];
        ah[mt][1] = Ah[(r + 8) * kALd + ks + tig];
        ah[mt][2] = Ah[r * kALd + ks + tig + 4];
        ah[mt][3] = Ah[(r + 8) * kALd + ks + tig + 4];
        al[mt][0] = Al[r * kALd + ks + tig];
        al[mt][1] = Al[(r + 8) * kALd + ks + tig];
        al[mt][2] = Al[r * kALd + ks + tig + 4];
        al[mt][3] = Al[(r + 8) * kALd + ks + tig + 4];
      }
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int cidx = wn + nt * 8 + gid;
        bh[nt][0] = Bh[(ks + tig) * kBLd + cidx];
        bh[nt][1] = Bh[(ks + tig + 4) * kBLd + cidx];
        bl[nt][0] = Bl[(ks + tig) * kBLd + cidx];
        bl[nt][1] = Bl[(ks + tig + 4) * kBLd + cidx];
      }
      // small products first, the chains of the eight tiles interleaved
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) mma_tf32(part[mt][nt], al[mt], bh[nt]);
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) mma_tf32(part[mt][nt], ah[mt], bl[nt]);
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) mma_tf32(part[mt][nt], ah[mt], bh[nt]);
    }
    // compensated addition of this chunk's result
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float y = part[i][j][e] - cmp[i][j][e];
          const float s = acc[i][j][e] + y;
          cmp[i][j][e] = (s - acc[i][j][e]) - y;
          acc[i][j][e] = s;
        }
    __syncthreads();
    jt = njt;
    k0 = nk0;
    g = ng;
  }
  TC* C = static_cast<TC*>(b.p[t.C.base]) + t.C.off;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = tl.m0 + wm + mt * 16 + gid + (e >= 2 ? 8 : 0);
        const int c = tl.n0 + wn + nt * 8 + 2 * tig + (e & 1);
        if (r < t.M && c < t.N) {
          TC* p = C + int64_t(r) * t.C.ld + c;
          *p = beta_zero ? TC(acc[mt][nt][e]) : TC(*p + TC(acc[mt][nt][e]));
        }
      }
}

// tasks of at most 1024 outputs: one warp each, FP32 FMAs on the CUDA cores
template <class TA, class TB, class TC>
__global__ void __launch_bounds__(256)
    k_gemm_small_f32(const GemmTask* __restrict__ tasks, int64_t n_tasks,
                     const GemmTerm* __restrict__ terms, Bases<void> b, int beta_zero,
                     const int32_t* __restrict__ active) {
  if (active && !active[0]) return;
  const int64_t w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  if (w >= n_tasks) return;
  const GemmTask t = tasks[w];
  TC* C = static_cast<TC*>(b.p[t.C.base]) + t.C.off;
  const int MN = t.M * t.N;
  for (int idx = lane; idx < MN; idx += 32) {
    const int m = idx / t.N, n = idx - m * t.N;
    // compensated (Kahan) summation of the products over k and terms
    float acc = 0.f, cmp = 0.f;
    for (int j = t.t0; j < t.t1; ++j) {
      const GemmTerm g = terms[j];
      const TA* A = static_cast<const TA*>(b.p[g.A.base]) + g.A.off;
      const TB* B = static_cast<const TB*>(b.p[g.B.base]) + g.B.off;
      const int ta = g.trans & 1, tb = (g.trans >> 1) & 1;
      const float alpha = float(g.alpha);
      for (int k = 0; k < g.K; ++k) {
        const float av = float(ta ? A[int64_t(k) * g.A.ld + m] : A[int64_t(m) * g.A.ld + k]);
        const float bv = float(tb ? B[int64_t(n) * g.B.ld + k] : B[int64_t(k) * g.B.ld + n]);
        const float pr = alpha * av * bv;
        const float y = pr - cmp;
        const float s = acc + y;
        cmp = (s - acc) - y;
        acc = s;
      }
    }
    TC* c = C + int64_t(m) * t.C.ld + n;
    *c = beta_zero ? TC(acc) : TC(*c + TC(acc));
  }
}

}  // namespace

template <class TA, class TB, class TC>
static void run_gemm_small_mixed(const DevTaskList& L, const Bases<void>& b, int beta_zero,
                                 cudaStream_t s, const int32_t* active) {
  const int64_t threads = L.n_small * 32;
  k_gemm_small_f32<TA, TB, TC><<<int((threads + 255) / 256), 256, 0, s>>>(
      L.small_tasks.p, L.n_small, L.terms.p, b, beta_zero, active);
  DMRG_LAUNCHED();
}

template <class TA, class TB, class TC>
void run_gemm_tasks_tc(const DevTaskList& L, const Bases<void>& b, int beta_zero,
                       cudaStream_t s, const int32_t* active) {
  static_assert(kTM == 64 && kTN == 64, "tiles of the task lists are 64 x 64");
  if (L.n_small) run_gemm_small_mixed<TA, TB, TC>(L, b, beta_zero, s, active);
  if (L.n_tiles) {
    k_gemm_tc<TA, TB, TC><<<int(L.n_tiles), kThreads, 0, s>>>(L.tiles.p, L.large_tasks.p,
                                                              L.terms.p, b, beta_zero, active);
    DMRG_LAUNCHED();
  }
}
template void run_gemm_tasks_tc<float, float, float>(const DevTaskList&, const Bases<void>&, int,
                                                     cudaStream_t, const int32_t*);
template void run_gemm_tasks_tc<double, double, float>(const DevTaskList&, const Bases<void>&,
                                                       int, cudaStream_t, const int32_t*);
template void run_gemm_tasks_tc<double, float, double>(const DevTaskList&, const Bases<void>&,
                                                       int, cudaStream_t, const int32_t*);

}  // namespace dmrg
